// footprint.cu -- csgv_footprint_*: the brick requests of one rendered frame (Sec. 4 of the paper,
// "Raymarching" and "Empty-Space Skipping").
//
// The paper's renderer marches one ray per pixel through the brick grid.  Each frame it first resets one
// integer per brick to "invisible"; a ray that passes a brick writes the level of detail it wants for
// that brick into the integer (every ray that reaches a brick computes the same LOD from the brick's
// distance, so the writes do not race), and a brick none of whose palette labels is opaque under the
// transfer function is skipped without a request (empty-space skipping).  The flagged bricks are then
// compacted into the frame's request list.
//
// Here, per frame:
//   footprint_march (one thread per pixel, 16 x 16 pixel tiles): the camera ray through the pixel centre
//     is clipped to the volume box and walked brick by brick (a 3D DDA on the brick grid).  Transfer
//     function: label 0 is transparent, every other label opaque.  A brick whose palette holds only
//     label 0 is skipped; any other brick is requested at LOD t = clamp(floor(log2(d / f_px)), 0, N)
//     (d: distance from the camera to the brick centre, f_px: focal length in pixels, so that one voxel
//     of the LOD covers about one pixel).  The ray stops at a brick whose root label (palette[0], the
//     mode of the whole brick) is opaque, or once it has requested max_nonempty bricks (0: no limit).
//   footprint_count / footprint_compact: the requested bricks in brick-id order (a count per 1024
//     bricks, then each block's offset and a block scan), with the per-brick integer reset to
//     "invisible" as it is read, ready for the next frame.
//
// Every float operation of the march is an explicitly rounded IEEE single-precision operation (no
// contraction into fused multiply-adds), so that a plain CPU restatement in float32 takes the same
// decisions; the LOD compares squared distances against (f_px 2^k)^2 instead of taking a logarithm.
#include <cstdio>

#include "csgv_internal.cuh"
#include "../../include/csgv.h"

namespace csgv {
void set_last_error(const char *msg);  // api.cu
VolDev volume_view(const csgv_volume *v);
cudaEvent_t volume_ready(const csgv_volume *v);
void volume_grid(const csgv_volume *v, uint64_t dims[3], uint64_t grid[3]);
}  // namespace csgv

struct csgv_footprint {
    const csgv_volume *vol;
    int dev;
    uint64_t n_bricks, dims[3], grid[3];
    uint32_t N, max_nonempty;
    uint8_t *flags = nullptr;   // per brick: bit 0 some palette label opaque, bit 1 palette[0] opaque
    int32_t *lod = nullptr;     // per brick: requested LOD this frame, -1 = invisible
    uint32_t *blk = nullptr;    // requests per 1024 bricks
};

namespace {

constexpr uint32_t kCompactBlock = 1024;
constexpr float kParallel = 1e-30f;  // |direction component| below this: the ray is parallel to that axis

int fail(int code, const char *msg) {
    csgv::set_last_error(msg);
    return code;
}
int cuda_fail(cudaError_t e, const char *what) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    csgv::set_last_error(buf);
    return CSGV_ERR_CUDA;
}

// per brick: bit 0 = the palette holds an opaque (non-zero) label, bit 1 = palette[0] is opaque
__global__ void brick_opacity(csgv::VolDev V, uint8_t *flags) {
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= V.n_bricks) return;
    const uint64_t p0 = V.pal_off[k], p1 = V.pal_off[k + 1];
    uint32_t any = 0;
    for (uint64_t j = p0; j < p1 && !any; j++) any = V.pal[j] != 0u;
    const uint32_t root = p1 > p0 && V.pal[p0] != 0u;
    flags[k] = (uint8_t)(any | (root << 1));
}

struct Ray {
    float o[3], right[3], up[3], fwd[3], f_px, half_w, half_h;
    float D[3];      // volume box [0, D)
    float B;         // brick side (a power of two)
    int G[3];        // bricks per axis
    uint32_t W, H, N, max_nonempty;
    uint64_t n_bricks;
};

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }

__global__ void __launch_bounds__(256) footprint_march(Ray R, const uint8_t *__restrict__ flags, int32_t *lod) {
    const uint32_t x = blockIdx.x * 16 + (threadIdx.x & 15), y = blockIdx.y * 16 + (threadIdx.x >> 4);
    if (x >= R.W || y >= R.H) return;
    // direction through the pixel centre (not normalised: the walk only compares ray parameters)
    const float px = fdiv(fsub(fadd((float)x, 0.5f), R.half_w), R.f_px);
    const float py = fdiv(fsub(fadd((float)y, 0.5f), R.half_h), R.f_px);
    float d[3], inv[3];
    float tn = -INFINITY, tf = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        d[a] = fsub(fadd(R.fwd[a], fmul(px, R.right[a])), fmul(py, R.up[a]));
        if (fabsf(d[a]) < kParallel) {
            d[a] = 0.0f;
            inv[a] = 0.0f;
            if (R.o[a] < 0.0f || R.o[a] > R.D[a]) return;  // parallel to the slab and outside it
            continue;
        }
        inv[a] = fdiv(1.0f, d[a]);
        const float t0 = fmul(fsub(0.0f, R.o[a]), inv[a]), t1 = fmul(fsub(R.D[a], R.o[a]), inv[a]);
        tn = fmaxf(tn, fminf(t0, t1));
        tf = fminf(tf, fmaxf(t0, t1));
    }
    const float t = fmaxf(tn, 0.0f);
    if (!(tf >= t) || !(tf > 0.0f)) return;  // misses the volume
    int idx[3], step[3];
    float tmax[3], tdel[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float p = fadd(R.o[a], fmul(d[a], t));
        int i = (int)floorf(fdiv(p, R.B));
        idx[a] = i < 0 ? 0 : (i >= R.G[a] ? R.G[a] - 1 : i);
        step[a] = d[a] > 0.0f ? 1 : (d[a] < 0.0f ? -1 : 0);
        if (step[a] == 0) {
            tmax[a] = INFINITY;
            tdel[a] = INFINITY;
        } else {
            const float bound = (float)((idx[a] + (step[a] > 0 ? 1 : 0)) * (int)R.B);
            tmax[a] = fmul(fsub(bound, R.o[a]), inv[a]);
            tdel[a] = fmul(R.B, fabsf(inv[a]));
        }
    }
    // LOD thresholds: t >= k iff d^2 >= (f_px 2^k)^2 (exact power-of-two scalings)
    uint32_t hits = 0;
    const int max_steps = R.G[0] + R.G[1] + R.G[2] + 3;
    for (int s = 0; s < max_steps; s++) {
        const uint64_t k = (uint64_t)idx[0] + (uint64_t)R.G[0] * ((uint64_t)idx[1] + (uint64_t)R.G[1] * idx[2]);
        const uint32_t fl = __ldg(flags + k);
        if (fl & 1u) {  // not empty: request it
            float d2 = 0.0f;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const float c = fmul(fadd((float)idx[a], 0.5f), R.B);
                const float e = fsub(c, R.o[a]);
                d2 = fadd(d2, fmul(e, e));
            }
            uint32_t lv = 0;
            float thr = R.f_px;
            for (uint32_t q = 1; q <= R.N; q++) {
                thr = fmul(thr, 2.0f);
                lv += d2 >= fmul(thr, thr) ? 1u : 0u;
            }
            if (lod[k] != (int32_t)lv) lod[k] = (int32_t)lv;  // every ray computes the same LOD for brick k
            hits++;
            if ((fl & 2u) || (R.max_nonempty && hits >= R.max_nonempty)) return;
        }
        // next brick: the axis whose boundary comes first (ties: lowest axis)
        int a = 0;
        if (tmax[1] < tmax[a]) a = 1;
        if (tmax[2] < tmax[a]) a = 2;
        if (tmax[a] > tf) return;  // leaves the volume
        idx[a] += step[a];
        if (idx[a] < 0 || idx[a] >= R.G[a]) return;
        tmax[a] = fadd(tmax[a], tdel[a]);
    }
}

// requests per block of kCompactBlock bricks
__global__ void __launch_bounds__(kCompactBlock) footprint_count(const int32_t *lod, uint64_t n, uint32_t *blk) {
    const uint64_t k = (uint64_t)blockIdx.x * kCompactBlock + threadIdx.x;
    const bool on = k < n && lod[k] >= 0;
    const uint32_t c = __syncthreads_count(on);
    if (threadIdx.x == 0) blk[blockIdx.x] = c;
}

// the requests of each block at its offset (sum of the earlier blocks' counts), in brick order; the
// per-brick LODs are reset to -1 (invisible) for the next frame
__global__ void __launch_bounds__(kCompactBlock) footprint_compact(int32_t *lod, uint64_t n, const uint32_t *blk,
                                                                   uint32_t *bricks, uint8_t *lods,
                                                                   uint32_t *n_out) {
    __shared__ uint32_t red[kCompactBlock / 32];
    __shared__ uint32_t base_s;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // offset of this block
    uint32_t part = 0;
    for (uint32_t j = tid; j < blockIdx.x; j += kCompactBlock) part += blk[j];
    for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(csgv::kFull, part, o);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = red[lane];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(csgv::kFull, v, o);
        if (lane == 0) base_s = v;
    }
    __syncthreads();
    const uint32_t base = base_s;
    // block scan of the flags
    const uint64_t k = (uint64_t)blockIdx.x * kCompactBlock + tid;
    const int32_t lv = k < n ? lod[k] : -1;
    const bool on = lv >= 0;
    const uint32_t m = __ballot_sync(csgv::kFull, on);
    __syncthreads();
    if (lane == 0) red[warp] = __popc(m);
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = red[lane];
        uint32_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(csgv::kFull, incl, o);
            if (lane >= (uint32_t)o) incl += u;
        }
        red[lane] = incl - v;
    }
    __syncthreads();
    if (on) {
        const uint32_t r = base + red[warp] + __popc(m & ((1u << lane) - 1u));
        bricks[r] = (uint32_t)k;
        lods[r] = (uint8_t)lv;
        lod[k] = -1;
    }
    if (blockIdx.x == gridDim.x - 1 && tid == 0) *n_out = base + blk[blockIdx.x];
}

}  // namespace

extern "C" {

int csgv_footprint_create(const csgv_volume *vol, uint32_t max_nonempty, csgv_footprint **out, void *stream) {
    if (!vol || !out) return fail(CSGV_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    csgv_footprint *fp = new csgv_footprint();
    fp->vol = vol;
    fp->max_nonempty = max_nonempty;
    const csgv::VolDev V = csgv::volume_view(vol);
    fp->n_bricks = V.n_bricks;
    fp->N = V.N;
    csgv::volume_grid(vol, fp->dims, fp->grid);
    if (fp->n_bricks == 0 || fp->n_bricks > 0xFFFFFFFFull) {
        delete fp;
        return fail(CSGV_ERR_INVALID_ARG, "volume must have 1 .. 2^32 - 1 bricks");
    }
    const uint64_t n_blk = (fp->n_bricks + kCompactBlock - 1) / kCompactBlock;
    cudaError_t e = cudaGetDevice(&fp->dev);
    if (e == cudaSuccess) e = cudaMalloc(&fp->flags, fp->n_bricks);
    if (e == cudaSuccess) e = cudaMalloc(&fp->lod, fp->n_bricks * 4);
    if (e == cudaSuccess) e = cudaMalloc(&fp->blk, n_blk * 4);
    cudaEvent_t ready = csgv::volume_ready(vol);
    if (e == cudaSuccess && ready) e = cudaStreamWaitEvent(st, ready, 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(fp->lod, 0xFF, fp->n_bricks * 4, st);  // every brick invisible
    if (e == cudaSuccess) {
        brick_opacity<<<(unsigned)((fp->n_bricks + 255) / 256), 256, 0, st>>>(V, fp->flags);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaFree(fp->flags);
        cudaFree(fp->lod);
        cudaFree(fp->blk);
        delete fp;
        return cuda_fail(e, "csgv_footprint_create");
    }
    *out = fp;
    return CSGV_OK;
}

int csgv_footprint_frame(csgv_footprint *fp, const csgv_camera *cam, uint32_t *bricks_dev, uint8_t *lods_dev,
                         uint32_t *n_dev, void *stream) {
    if (!fp || !cam || !bricks_dev || !lods_dev || !n_dev) return fail(CSGV_ERR_INVALID_ARG, "NULL argument");
    if (cam->width == 0 || cam->height == 0 || cam->width > 65536 || cam->height > 65536 || !(cam->f_px > 0.0f))
        return fail(CSGV_ERR_INVALID_ARG, "camera: width and height must be 1..65536 and f_px > 0");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != fp->dev)
        return fail(CSGV_ERR_INVALID_ARG, "the footprint belongs to another device");
    cudaStream_t st = (cudaStream_t)stream;
    Ray R;
    for (int a = 0; a < 3; a++) {
        R.o[a] = cam->pos[a];
        R.right[a] = cam->right[a];
        R.up[a] = cam->up[a];
        R.fwd[a] = cam->fwd[a];
        R.D[a] = (float)fp->dims[a];
        R.G[a] = (int)fp->grid[a];
    }
    R.f_px = cam->f_px;
    R.half_w = 0.5f * (float)cam->width;
    R.half_h = 0.5f * (float)cam->height;
    R.B = (float)(1u << fp->N);
    R.W = cam->width;
    R.H = cam->height;
    R.N = fp->N;
    R.max_nonempty = fp->max_nonempty;
    R.n_bricks = fp->n_bricks;
    const dim3 grid((cam->width + 15) / 16, (cam->height + 15) / 16);
    {
        csgv::ProfScope ps("footprint_march", st);
        footprint_march<<<grid, 256, 0, st>>>(R, fp->flags, fp->lod);
    }
    const uint64_t n_blk = (fp->n_bricks + kCompactBlock - 1) / kCompactBlock;
    {
        csgv::ProfScope ps("footprint_compact", st);
        footprint_count<<<(unsigned)n_blk, kCompactBlock, 0, st>>>(fp->lod, fp->n_bricks, fp->blk);
        footprint_compact<<<(unsigned)n_blk, kCompactBlock, 0, st>>>(fp->lod, fp->n_bricks, fp->blk, bricks_dev,
                                                                      lods_dev, n_dev);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CSGV_OK : cuda_fail(e, "csgv_footprint_frame");
}

int csgv_footprint_destroy(csgv_footprint *fp) {
    if (!fp) return CSGV_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != fp->dev) cudaSetDevice(fp->dev);
    cudaFree(fp->flags);
    cudaFree(fp->lod);
    cudaFree(fp->blk);
    if (prev >= 0 && prev != fp->dev) cudaSetDevice(prev);
    delete fp;
    return CSGV_OK;
}

}  // extern "C"
