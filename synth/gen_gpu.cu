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


// ---- fibers: the generator of gen.c (synth_fibers), brick by brick; same integer formulas
constexpr int kFibBalls = 16, kFibMargin = 32, kFibReach = 48;
constexpr uint32_t kFibThreads = 512, kFibTubesPerRound = 128;

__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t d) { return a >= 0 ? a / d : -((-a + d - 1) / d); }
__device__ __forceinline__ uint64_t fib_hash(uint64_t seed, uint64_t t, uint64_t j) {
    return hash2(seed ^ 0xF1BE5ull, t * 16 + j);
}
__device__ __forceinline__ int64_t isqrt64(int64_t n) {
    int64_t w = (int64_t)sqrt((double)n);
    while (w * w > n) w--;
    while ((w + 1) * (w + 1) <= n) w++;
    return w;
}

struct FibBall {
    int16_t c[3];  // centre relative to the brick origin, 1/8-voxel units
    uint16_t r;    // radius, 1/8-voxel units
    uint32_t t;    // tube id
};

// One CTA per brick: gather the balls of the tubes that can reach the brick (cells within kFibReach voxels),
// then take the lowest tube id per voxel in shared memory and write the brick's labels (b^3, x fastest).
__global__ void __launch_bounds__(kFibThreads) fiber_bricks_kernel(uint32_t *out, const uint64_t *ids, uint64_t first,
                                                                   uint64_t X, uint64_t Y, uint64_t Z, uint32_t b,
                                                                   int64_t G, uint32_t T, uint64_t seed) {
    extern __shared__ __align__(16) uint32_t key[];            // b^3 lowest tube ids
    FibBall *balls = reinterpret_cast<FibBall *>(key + (size_t)b * b * b);  // kFibTubesPerRound * 2 * kFibBalls
    __shared__ uint32_t nballs;
    const uint64_t id = ids ? ids[blockIdx.x] : first + blockIdx.x;
    const uint64_t nbx = (X + b - 1) / b, nby = (Y + b - 1) / b;
    const int64_t B0[3] = {(int64_t)((id % nbx) * b), (int64_t)(((id / nbx) % nby) * b), (int64_t)((id / (nbx * nby)) * b)};
    const int64_t dims[3] = {(int64_t)X, (int64_t)Y, (int64_t)Z};
    const uint64_t nc[3] = {(X + G - 1) / G, (Y + G - 1) / G, (Z + G - 1) / G};
    int64_t clo[3], cn[3];
    for (int a = 0; a < 3; a++) {
        int64_t lo = floor_div(B0[a] - kFibReach, G), hi = floor_div(B0[a] + b - 1 + kFibReach, G);
        lo = lo < 0 ? 0 : lo;
        hi = hi > (int64_t)nc[a] - 1 ? (int64_t)nc[a] - 1 : hi;
        clo[a] = lo;
        cn[a] = hi - lo + 1;
    }
    const uint32_t ntubes = (uint32_t)(cn[0] * cn[1] * cn[2]) * T;
    const uint32_t nvox = b * b * b;
    for (uint32_t i = threadIdx.x; i < nvox; i += blockDim.x) key[i] = 0xFFFFFFFFu;
    for (uint32_t r0 = 0; r0 < ntubes; r0 += kFibTubesPerRound) {
        if (threadIdx.x == 0) nballs = 0;
        __syncthreads();
        // the balls of this round's tubes that reach the brick (one thread per tube)
        for (uint32_t j = r0 + threadIdx.x; j < min(ntubes, r0 + kFibTubesPerRound); j += blockDim.x) {
            const uint32_t k = j % T, cl = j / T;
            const int64_t cc[3] = {clo[0] + (int64_t)(cl % cn[0]), clo[1] + (int64_t)((cl / cn[0]) % cn[1]),
                                   clo[2] + (int64_t)(cl / (cn[0] * cn[1]))};
            const uint64_t t = ((uint64_t)cc[0] + nc[0] * ((uint64_t)cc[1] + nc[1] * (uint64_t)cc[2])) * T + k;
            const int64_t O[3] = {cc[0] * G, cc[1] * G, cc[2] * G};
            const uint64_t h0 = fib_hash(seed, t, 0), h1 = fib_hash(seed, t, 1);
            int64_t P[5][3], D[3];
            for (int a = 0; a < 3; a++) {
                P[0][a] = O[a] + (int64_t)(((h0 >> (16 * a)) & 0xFFFFull) % (uint64_t)G);
                D[a] = (int64_t)((h1 >> (8 * a)) & 15ull) - 8;
            }
            for (int i = 1; i < 5; i++) {
                const uint64_t h = fib_hash(seed, t, 1 + i);
                for (int a = 0; a < 3; a++) {
                    const int64_t p = P[i - 1][a] + D[a] + (int64_t)((h >> (8 * a)) & 7ull) - 4;
                    const int64_t lo = O[a] - kFibMargin, hi = O[a] + G + kFibMargin - 1;
                    P[i][a] = p < lo ? lo : (p > hi ? hi : p);
                }
            }
            const int64_t R = 8 * (2 + (int64_t)(fib_hash(seed, t, 6) % 5));
            for (int span = 1; span <= 2; span++)
                for (int64_t q = 0; q < kFibBalls; q++) {
                    int64_t c[3];
                    bool hit = true;
                    for (int a = 0; a < 3; a++) {
                        const int64_t p0 = P[span - 1][a], p1 = P[span][a], p2 = P[span + 1][a], p3 = P[span + 2][a];
                        const int64_t A = p2 - p0, Bq = 2 * p0 - 5 * p1 + 4 * p2 - p3, Cc = -p0 + 3 * p1 - 3 * p2 + p3;
                        c[a] = floor_div(8192 * p1 + 256 * A * q + 16 * Bq * q * q + Cc * q * q * q, 1024);
                        // voxels of the ball along a: ceil((c - 4 - R) / 8) .. floor((c - 4 + R) / 8), inside the
                        // brick and the volume
                        const int64_t lo = -floor_div(-(c[a] - 4 - R), 8), hi = floor_div(c[a] - 4 + R, 8);
                        const int64_t blo = B0[a], bhi = min(B0[a] + (int64_t)b, dims[a]) - 1;
                        hit = hit && lo <= bhi && hi >= blo;
                    }
                    if (hit) {
                        const uint32_t at = atomicAdd(&nballs, 1u);
                        FibBall f;
                        for (int a = 0; a < 3; a++) f.c[a] = (int16_t)(c[a] - 8 * B0[a]);
                        f.r = (uint16_t)R;
                        f.t = (uint32_t)t;
                        balls[at] = f;
                    }
                }
        }
        __syncthreads();
        // each ball: its rows inside the brick, the x run of each row from an exact integer square root
        const uint32_t nb_ = nballs;
        for (uint32_t j = threadIdx.x; j < nb_; j += blockDim.x) {
            const FibBall f = balls[j];
            const int64_t R = f.r;
            int64_t lo[3], hi[3];
            for (int a = 0; a < 3; a++) {
                lo[a] = -floor_div(-((int64_t)f.c[a] - 4 - R), 8);
                hi[a] = floor_div((int64_t)f.c[a] - 4 + R, 8);
                const int64_t lim = min((int64_t)b, dims[a] - B0[a]) - 1;
                lo[a] = lo[a] < 0 ? 0 : lo[a];
                hi[a] = hi[a] > lim ? lim : hi[a];
            }
            for (int64_t z = lo[2]; z <= hi[2]; z++) {
                const int64_t dz = 8 * z + 4 - f.c[2];
                for (int64_t y = lo[1]; y <= hi[1]; y++) {
                    const int64_t dy = 8 * y + 4 - f.c[1], rem = R * R - dz * dz - dy * dy;
                    if (rem < 0) continue;
                    const int64_t w = isqrt64(rem);
                    int64_t x0 = -floor_div(-((int64_t)f.c[0] - 4 - w), 8), x1 = floor_div((int64_t)f.c[0] - 4 + w, 8);
                    x0 = x0 < lo[0] ? lo[0] : x0;
                    x1 = x1 > hi[0] ? hi[0] : x1;
                    for (int64_t x = x0; x <= x1; x++) atomicMin(&key[x + b * (y + b * z)], f.t);
                }
            }
        }
        __syncthreads();
    }
    uint32_t *o = out + (size_t)blockIdx.x * nvox;
    for (uint32_t i = threadIdx.x; i < nvox; i += blockDim.x)
        o[i] = key[i] == 0xFFFFFFFFu ? 0u : label_of(seed ^ 0xF1BE5ull, key[i]);
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

// Bricks of the fiber volume (synth_fibers of gen.c) without the volume: brick ids first .. first + m - 1, or
// ids_dev[0 .. m - 1] when given, each as b^3 labels (x fastest) at out_dev + i * b^3.  Bricks must lie inside
// the volume (dims multiples of b).  b <= 32.
extern "C" __attribute__((visibility("default"))) int synth_fiber_bricks_dev(uint32_t *out_dev, const uint64_t *ids_dev,
                                                                             uint64_t first, uint32_t m, uint64_t X,
                                                                             uint64_t Y, uint64_t Z, uint32_t b,
                                                                             uint32_t cell, uint32_t tubes,
                                                                             uint64_t seed, void *stream) {
    if (!out_dev || !cell || !tubes || !b || b > 32 || X % b || Y % b || Z % b) return 1;
    if (m == 0) return 0;
    const size_t smem = (size_t)b * b * b * 4 + (size_t)kFibTubesPerRound * 2 * kFibBalls * sizeof(FibBall);
    if (cudaFuncSetAttribute(fiber_bricks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 2;
    fiber_bricks_kernel<<<m, kFibThreads, smem, (cudaStream_t)stream>>>(out_dev, ids_dev, first, X, Y, Z, b, cell,
                                                                       tubes, seed);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
