/*
 * csgv.h -- C ABI of libcsgv.so, a B300 (sm_103a) implementation of the
 * compressed segmentation volume brick codec of Piochowiak & Dachsbacher,
 * "Fast Compressed Segmentation Volumes for Scientific Visualization"
 * (IEEE TVCG 2023).
 *
 * Conventions for every call:
 *   - Pointers named *_dev are CUDA device pointers owned by the caller
 *     unless stated otherwise; *_host are host pointers.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on it unless stated otherwise.
 *   - Volumes are uint32 labels, x fastest: element (x, y, z) at
 *     x + dims[0] * (y + dims[1] * z).
 *   - Return value: CSGV_OK or an error code; csgv_last_error() gives a
 *     message for the calling thread.  No call throws, and no kernel traps:
 *     corrupt data is reported through status words.
 *
 * Stream format (fixed readings of the paper, Sec. 3):
 *   brick b = 2^N (N = 1..6), clamp-to-edge padding, brick id
 *   bx + nbx * (by + nby * bz); per brick a palette of uint32 labels and two
 *   rANS-coded nibble streams (interior: children on levels N-1..1; leaf:
 *   children on level 0).  Nibble = op | stop << 3 with R_p=0 R_x=1 R_y=2
 *   R_z=3 P_0=4 P_delta=5 P_a=6, a P_delta nibble followed by its delta.
 *   rANS: 32-bit states, M = 4096, L = 2^16, 16-bit words; K =
 *   clamp(n / S_min, 1, K_max) interleaved states; stream = K final states
 *   (low half first) then renormalisation words in decode order.
 */
#ifndef CSGV_H
#define CSGV_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CSGV_API __attribute__((visibility("default")))
#else
#define CSGV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CSGV_OK = 0,
    CSGV_PENDING = 1,          /* serve: ticket not finished yet */
    CSGV_ERR_INVALID_ARG = 2,  /* bad argument (host-side check) */
    CSGV_ERR_OOM = 3,          /* device or host allocation failed */
    CSGV_ERR_CORRUPT = 4,      /* per-request status: stream does not follow the format */
    CSGV_ERR_TIMEOUT = 5,      /* a bounded wait ran out */
    CSGV_ERR_CUDA = 6,         /* a CUDA runtime call failed */
    CSGV_ERR_RANGE = 7         /* per-request status: brick id or LOD out of range */
};

/* Two static nibble frequency tables (Sec. 3.3): interior then leaf, each
 * 16 entries summing to 4096, every entry >= 1. */
typedef struct {
    uint32_t freq[32];
    uint64_t counts[32]; /* raw nibble counts of the prepass (diagnostic) */
} csgv_freq_table;

/* Encoder parameters (interleaving rule R10). */
typedef struct {
    uint32_t K_max; /* most interleaved rANS states per stream, 1..32 (default 32) */
    uint32_t S_min; /* symbols per state before another state is added (default 256) */
} csgv_config;

typedef struct csgv_volume csgv_volume;

typedef struct {
    uint32_t N;             /* log2 brick size */
    uint64_t dims[3];       /* volume size in voxels */
    uint64_t grid[3];       /* bricks per axis */
    uint64_t n_bricks;
    uint32_t K_max, S_min;
    uint32_t max_palette;   /* largest palette of any brick */
    uint64_t palette_labels, int_words, leaf_words;
    uint64_t compressed_bytes; /* palettes + streams + per-brick header (3 u64 offsets + 2 u32 counts) */
    uint32_t freq[32];
} csgv_volume_info;

/* Message of the last error on this thread ("" if none). */
CSGV_API const char *csgv_last_error(void);

/*
 * Frequency prepass (Sec. 3.3 and 3.4: the two frequency tables come from
 * the nibbles of a sample of the bricks, encoded beforehand).  Runs the brick
 * encoder in count-only mode over every brick whose id is a multiple of
 * sample_stride, counts interior and leaf nibbles, and normalises each
 * table to 4096 (f = 1 + floor(c * 4080 / total), remainder to the largest
 * counts).  vol_dev: dims[0]*dims[1]*dims[2] labels.  b: 2..64, a power of
 * two.  Synchronises `stream` (reads 32 counters back).
 */
CSGV_API int csgv_build_freq_table(const uint32_t *vol_dev, const uint64_t dims[3], uint32_t b, uint32_t sample_stride,
                          csgv_freq_table *out, void *stream);

/*
 * Tables from nibble counts (Sec. 3.3; normalisation as in csgv_build_freq_table): counts[0..15]
 * interior, counts[16..31] leaf.  For sharded volumes: every rank counts its bricks with
 * csgv_build_freq_table, the counts are summed across ranks, and this turns the sums into the shared
 * tables.  Host only; fills out->freq and copies the counts to out->counts.
 */
CSGV_API int csgv_freq_table_from_counts(const uint64_t counts[32], csgv_freq_table *out);

/*
 * Brick encoder (Alg. 2, Sec. 3.2-3.4) for every brick of the volume, then
 * entropy coding and packing.  The library allocates the compressed arrays;
 * the returned volume owns them until csgv_volume_destroy.  cfg may be NULL
 * (defaults).  Synchronises `stream` once per encode batch (reads the sizes
 * back to allocate), then packs asynchronously on it: the volume is complete
 * in the order of `stream`.  Decodes on other streams wait for it through an
 * event the library records (except inside a stream capture, which cannot
 * depend on uncaptured work: launch such a graph once the volume is complete);
 * csgv_volume_export and csgv_volume_destroy synchronise the device.
 */
CSGV_API int csgv_encode_bricks(const uint32_t *vol_dev, const uint64_t dims[3], uint32_t b, const csgv_freq_table *table,
                       const csgv_config *cfg, csgv_volume **out, void *stream);

/*
 * Prepass and encode in one call: the op streams of every brick are made first
 * (they do not depend on the tables), the nibbles of every sample_stride-th
 * brick are counted from them, the tables are normalised from those counts as
 * csgv_build_freq_table does, and the streams are then entropy-coded.  The
 * result is byte-identical to csgv_build_freq_table followed by
 * csgv_encode_bricks, without coding the sampled bricks twice.  *table_out
 * (if not NULL) receives the tables.  The counts, the tables and the coding
 * stay on the device; the call synchronises `stream` once, like
 * csgv_encode_bricks.  Volumes larger than one encode batch take the two-call
 * path internally.
 */
CSGV_API int csgv_encode_bricks_sampled(const uint32_t *vol_dev, const uint64_t dims[3], uint32_t b,
                                        uint32_t sample_stride, const csgv_config *cfg, csgv_freq_table *table_out,
                                        csgv_volume **out, void *stream);

/*
 * Batched decoding (Alg. 1, Sec. 4.1: all the bricks a frame needs, each at
 * its own level of detail, decoded on the GPU at once).  Request r decodes
 * brick brick_ids_dev[r] to level of detail lods_dev[r] (0 = full
 * resolution, N = the single root label) into out_dev + out_offsets_dev[r]:
 * (b >> lod)^3 labels, x fastest.  An offset may be any label index; outputs
 * that start on a 16-byte boundary take 16-byte stores, the others 8- or 4-byte
 * ones (the same bytes, more store instructions).  Per slice of requests (sized by the
 * workspace): a persistent rANS kernel whose warps take streams from a work
 * counter, then the reconstruction, one CTA per request (large mixed-LOD
 * slices: one persistent kernel per LOD class).  status_dev[r] receives CSGV_OK,
 * CSGV_ERR_CORRUPT or CSGV_ERR_RANGE.  All request arrays are device arrays
 * of n entries owned by the caller.  Asynchronous; the return value covers
 * argument and launch errors only.
 */
CSGV_API int csgv_decode_bricks(const csgv_volume *vol, const uint32_t *brick_ids_dev, const uint8_t *lods_dev, uint32_t n,
                       uint32_t *out_dev, const uint64_t *out_offsets_dev, int32_t *status_dev, void *stream);

/*
 * Same results as csgv_decode_bricks, one kernel launch per request (the
 * plain per-brick baseline).
 */
CSGV_API int csgv_decode_bricks_plain(const csgv_volume *vol, const uint32_t *brick_ids_dev, const uint8_t *lods_dev,
                             uint32_t n, uint32_t *out_dev, const uint64_t *out_offsets_dev, int32_t *status_dev,
                             void *stream);

/* Sizes and tables of a volume (host call, no device work). */
CSGV_API int csgv_volume_info_get(const csgv_volume *vol, csgv_volume_info *info);

/*
 * Copy the compressed arrays to host buffers sized from csgv_volume_info:
 * offsets have n_bricks + 1 entries (palette offsets in labels, word offsets
 * in 16-bit words), counts n_bricks entries.  Any pointer may be NULL to
 * skip that array.  Synchronous.
 */
CSGV_API int csgv_volume_export(const csgv_volume *vol, uint64_t *pal_off_host, uint32_t *pal_host, uint64_t *int_off_host,
                       uint16_t *int_words_host, uint64_t *leaf_off_host, uint16_t *leaf_words_host,
                       uint32_t *n_int_sym_host, uint32_t *n_leaf_sym_host);

/*
 * Build a device volume from host arrays in the layout of csgv_volume_export
 * (for example a stream written by another encoder, or loaded from disk).
 * freq: 32 entries.  Synchronous.
 */
CSGV_API int csgv_volume_import(uint32_t N, const uint64_t dims[3], uint32_t K_max, uint32_t S_min, const uint32_t freq[32],
                       const uint64_t *pal_off_host, const uint32_t *pal_host, const uint64_t *int_off_host,
                       const uint16_t *int_words_host, const uint64_t *leaf_off_host, const uint16_t *leaf_words_host,
                       const uint32_t *n_int_sym_host, const uint32_t *n_leaf_sym_host, csgv_volume **out);

/*
 * Streaming encoder: the volume's bricks arrive in batches from any source
 * (a procedural generator, a file read in pieces) and the raw volume never has
 * to exist in device memory as a whole.  A batch is m whole bricks in
 * brick-major order: brick i of the batch is b^3 uint32 labels at
 * bricks_dev + i * b^3, x fastest within the brick, already padded (voxels
 * past the volume's edge carry the clamp-to-edge labels).  Batches must come
 * in brick-id order (first = the number of bricks added so far) and cover all
 * bricks before csgv_stream_encoder_finish.  The result is the same volume
 * csgv_encode_bricks makes from the whole raw volume with the same tables and
 * configuration.
 *
 * csgv_stream_encoder_create: dims, b and cfg as for csgv_encode_bricks; the
 * tables are required (see csgv_count_bricks for a prepass over sampled
 * bricks).  Asynchronous on `stream`.
 * csgv_stream_encoder_add: encodes the batch; the caller may reuse bricks_dev
 * once the call returns (it synchronises `stream` once per internal batch).
 * csgv_stream_encoder_finish: hands over the completed volume (complete in the
 * order of `stream`) and frees the encoder.
 * csgv_stream_encoder_destroy: abandons an unfinished encoder (synchronises the
 * device).
 */
typedef struct csgv_stream_encoder csgv_stream_encoder;
CSGV_API int csgv_stream_encoder_create(const uint64_t dims[3], uint32_t b, const csgv_freq_table *table,
                                        const csgv_config *cfg, csgv_stream_encoder **out, void *stream);
CSGV_API int csgv_stream_encoder_add(csgv_stream_encoder *enc, const uint32_t *bricks_dev, uint64_t first,
                                     uint32_t m, void *stream);
CSGV_API int csgv_stream_encoder_finish(csgv_stream_encoder *enc, csgv_volume **out, void *stream);
CSGV_API void csgv_stream_encoder_destroy(csgv_stream_encoder *enc);

/*
 * Frequency prepass over a batch of bricks in the layout of
 * csgv_stream_encoder_add (m bricks of b^3 labels, brick-major): adds the
 * batch's 2 x 16 nibble counts to counts[0..31] (host, in/out), for
 * csgv_freq_table_from_counts.  Synchronises `stream`.
 */
CSGV_API int csgv_count_bricks(const uint32_t *bricks_dev, uint32_t m, uint32_t b, uint64_t counts[32],
                               void *stream);

/*
 * Allocation-free brick encoder, for callers that cannot call cudaMalloc:
 * programs whose device memory belongs to their own pool allocator, and
 * loops that cannot afford cudaFree's device-wide synchronisation.  The
 * paper has no counterpart; it is the encoder of csgv_encode_bricks
 * (same kernels, byte-identical output) working in a fixed 32 MiB scratch
 * array that the library keeps on every GPU that loads it, and writing into
 * device arrays the caller provides, in the layout of csgv_volume_export:
 * offsets with n_bricks + 1 entries (u64), palettes (u32), interior and leaf
 * words (u16), symbol counts (u32, n_bricks).  *_capacity give the sizes of
 * pal_dev, int_words_dev and leaf_words_dev in elements.
 * Limits: at most 99 bricks of 32^3 (11 of 64^3, 790 of 16^3, 6004 of 8^3,
 * 29025 of 4^3, 52101 of 2^3) per call; larger volumes are rejected with
 * CSGV_ERR_INVALID_ARG and a message.  totals[3] (host) receives the number of
 * palette labels, interior words and leaf words; if an output array is too
 * small the call returns CSGV_ERR_INVALID_ARG with totals filled and writes
 * nothing past the offset arrays.  Synchronises `stream` once (to read the
 * totals), then packs asynchronously on it.
 * Every call shares the scratch array, which keeps the previous call's
 * contents (the call clears what must start at zero); calls that overlap on
 * the GPU race on it and must not be issued.  The first call on a device,
 * made with that device current, looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.
 */
CSGV_API int csgv_encode_bricks_noalloc(const uint32_t *vol_dev, const uint64_t dims[3], uint32_t b,
                                        const csgv_freq_table *table, const csgv_config *cfg, uint64_t *pal_off_dev,
                                        uint32_t *pal_dev, uint64_t pal_capacity, uint64_t *int_off_dev,
                                        uint16_t *int_words_dev, uint64_t int_capacity, uint64_t *leaf_off_dev,
                                        uint16_t *leaf_words_dev, uint64_t leaf_capacity, uint32_t *n_int_sym_dev,
                                        uint32_t *n_leaf_sym_dev, uint64_t totals[3], void *stream);

/* ---------------------------------------------------------------- serving (Sec. 4.1) */

typedef struct csgv_server csgv_server;

typedef struct {
    uint64_t cache_bytes; /* decoded-brick cache in device memory (0: 8 GiB) */
    uint32_t max_batch;   /* most requests per decode launch (0: 16384) */
    uint32_t n_streams;   /* CUDA streams for overlapping batches (0: 3, at most 16) */
} csgv_serve_config;

typedef struct {
    const uint32_t *labels_dev; /* (b >> lod)^3 labels, x fastest, inside the cache; NULL on error */
    int32_t status;             /* CSGV_OK, CSGV_ERR_CORRUPT or CSGV_ERR_RANGE */
    uint32_t brick;
    uint8_t lod;
    uint8_t pad[3];
} csgv_result;

typedef struct {
    uint64_t submitted, hits, shared, misses, evictions, rebuilds, batches, decoded_labels;
    uint64_t cache_labels_used, cache_entries;
} csgv_serve_stats;

/*
 * Start a decode server for `vol` (which must outlive it): a cache of decoded
 * bricks in device memory and a worker thread.  Requests are deduplicated
 * against the cache (hits are served from it; a brick being decoded for
 * another ticket is shared), misses are admitted while cache space can be
 * found (free slot of the LOD's size, fresh space, least recently used
 * unpinned entry of the same LOD, or a rebuild when nothing is pinned) and
 * decoded in batches, one persistent launch each, round-robin over several
 * streams, so work submitted while other batches run overlaps on the device.
 * All requests of one ticket must fit in the cache together.
 */
CSGV_API int csgv_serve_create(const csgv_volume *vol, const csgv_serve_config *cfg, csgv_server **out);

/* Queue n requests (host arrays: brick ids, LODs); *ticket identifies them.  Never blocks on the GPU. */
CSGV_API int csgv_serve_submit(csgv_server *s, const uint32_t *bricks_host, const uint8_t *lods_host, uint32_t n,
                               uint64_t *ticket);

/*
 * Wait up to timeout_us for a ticket: CSGV_OK when every request is decoded
 * (results[n] filled, in submit order), CSGV_PENDING when timeout_us == 0 and
 * it is not finished, CSGV_ERR_TIMEOUT when the wait ran out.  Results point
 * into the cache and stay valid until csgv_serve_release.
 */
CSGV_API int csgv_serve_poll(csgv_server *s, uint64_t ticket, uint32_t timeout_us, csgv_result *results);

/* Unpin a finished ticket's cache entries (they become evictable) and forget the ticket. */
CSGV_API int csgv_serve_release(csgv_server *s, uint64_t ticket);

/* Counters, and the submit-to-completion latency (ms) of finished tickets in completion order. */
CSGV_API int csgv_serve_stats_get(csgv_server *s, csgv_serve_stats *out, double *latency_ms_host,
                                  uint32_t max_latencies, uint32_t *n_latencies);

/* Stop the worker, wait for batches in flight, free the cache. */
CSGV_API void csgv_serve_destroy(csgv_server *s);

/* ------------------------------------------- request footprint of a frame (Sec. 4, raymarching) */

/*
 * A pinhole camera in voxel units (the volume spans [0, dims) on each axis):
 * position, an orthonormal basis (right, up, forward; image rows grow
 * downward, along -up) and the focal length in pixels.  Pixel (x, y) looks
 * along fwd + px right - py up with px = (x + 0.5 - width / 2) / f_px and
 * py = (y + 0.5 - height / 2) / f_px.
 */
typedef struct {
    float pos[3], right[3], up[3], fwd[3];
    float f_px;
    uint32_t width, height;
} csgv_camera;

typedef struct csgv_footprint csgv_footprint;

/*
 * State for the brick requests of rendered frames of `vol` (which must
 * outlive it), after the paper's renderer (Sec. 4, "Raymarching" and
 * "Empty-Space Skipping"): one integer per brick, reset to "invisible"
 * each frame, into which the rays write the LOD they request.  The transfer
 * function maps label 0 to transparent and every other label to opaque; a
 * brick whose palette holds no opaque label is skipped without a request.
 * Each ray stops at a brick whose root label (palette[0]) is opaque, or once
 * it has requested max_nonempty bricks (0 = no such limit; 1 = the first
 * brick that holds an opaque label).  Allocates n_bricks * 5 bytes of device
 * memory plus 4 bytes per 1024 bricks; the per-brick flags are computed from
 * the palettes on `stream`.  Returns CSGV_ERR_INVALID_ARG for NULL arguments,
 * CSGV_ERR_CUDA if an allocation or launch fails.
 */
CSGV_API int csgv_footprint_create(const csgv_volume *vol, uint32_t max_nonempty, csgv_footprint **out,
                                   void *stream);

/*
 * One frame: every pixel's ray walks the brick grid (3D DDA, from where it
 * enters the volume box) and requests each brick it passes that holds an
 * opaque label, at LOD clamp(floor(log2(d / f_px)), 0, N), d the distance
 * from the camera to the brick centre; then the requests are written in
 * brick-id order to bricks_dev / lods_dev (capacity: n_bricks each) and
 * their number to *n_dev (device), and the per-brick integers are reset for
 * the next frame.  Float arithmetic is IEEE single precision with every
 * operation rounded on its own (no fused multiply-adds).  Asynchronous on
 * `stream`; successive frames of one footprint must be ordered (one stream).
 */
CSGV_API int csgv_footprint_frame(csgv_footprint *fp, const csgv_camera *cam, uint32_t *bricks_dev,
                                  uint8_t *lods_dev, uint32_t *n_dev, void *stream);

/* Free the footprint's device memory (synchronous). */
CSGV_API int csgv_footprint_destroy(csgv_footprint *fp);

/* Free a volume and its device arrays (synchronises the device). */
CSGV_API void csgv_volume_destroy(csgv_volume *vol);

/*
 * Free a volume in stream order, without synchronising: its device arrays are
 * released on `stream` once the work queued there before this call is done
 * (and once the volume itself is complete, if it was made on another stream).
 * Every call that uses the volume must already be queued on `stream`, or be
 * ordered before it; the handle is invalid on return.  A volume whose leaf
 * words are in host memory (csgv_volume_leaves_to_host) is freed as by
 * csgv_volume_destroy.  Returns CSGV_ERR_CUDA if a free could not be queued
 * (the volume is freed all the same).
 */
CSGV_API int csgv_volume_destroy_async(csgv_volume *vol, void *stream);

/*
 * Detail separation (Sec. 4.2 of the paper): move the leaf streams (the data of
 * level 0, about two thirds of the compressed words) to page-locked host
 * memory that the GPU maps, and free their device copy.  Decoding then reads
 * them in place over the host link when a request needs LOD 0; coarser LODs
 * never touch them.  Returns CSGV_ERR_OOM if the host allocation fails.
 * csgv_volume_leaves_to_device moves them back.  Both synchronise the device.
 */
CSGV_API int csgv_volume_leaves_to_host(csgv_volume *vol);
CSGV_API int csgv_volume_leaves_to_device(csgv_volume *vol);

/*
 * The launch shape of a volume's decodes (csgv_decode_autotune picks it; it
 * changes speed only, never the decoded labels).  Defaults: 192 MiB, 4, 512,
 * 128, 128, 1280 (the fastest point for 4096 LOD 0 requests of 32^3 bricks).
 */
typedef struct csgv_decode_tuning {
    uint64_t workspace_bytes;  /* op-record workspace per slice of requests (more: fewer, larger slices) */
    uint32_t rans_ctas_per_sm; /* CTAs (8 warps each) per SM of the rANS record kernel: 4, 5 or 6 */
    uint32_t ring_words;       /* stream words each rANS warp stages in shared memory: 128, 256 or 512
                                  (512 allows at most 5 CTAs per SM) */
    uint32_t rebuild_threads;  /* threads (warps x 32) per LOD 0 request of a 32^3 brick: 128 or 256 */
    uint32_t medium_threads;   /* threads per LOD 1 request of a 32^3 brick in batches of 8192 or more
                                  requests: 64, 128 or 256 */
    uint32_t compact_nodes;    /* a LOD 0 request of a 32^3 brick with at most this many non-constant L1
                                  nodes is rebuilt in the compact layout (rebuild_threads threads), one with
                                  more in the full layout (256 threads); 0 .. 1280 */
    uint32_t pad;
    double ms;                 /* measured time of the batch with this configuration (autotune only) */
} csgv_decode_tuning;

/*
 * Autotuner (batching at scale): time decode configurations on this batch and
 * keep the fastest in the volume for later csgv_decode_bricks calls; *best
 * receives it.  One knob at a time, each from the best point so far: rANS ring
 * depth x CTAs per SM, threads per LOD 0 request, the compact/full split of LOD
 * 0 requests (0, 256, 512, 1024, 1280 nodes), threads per LOD 1 request,
 * workspace per slice (64 MiB .. 1 GiB); each point is timed as the median of
 * five runs after a warm-up run (CUDA events on the stream).  The batch's
 * outputs are written by every run.  Synchronises the stream.  The paper has
 * no counterpart (it names work queues and batching as future work, Sec. 4.3).
 */
CSGV_API int csgv_decode_autotune(csgv_volume *vol, const uint32_t *brick_ids_dev, const uint8_t *lods_dev, uint32_t n,
                                  uint32_t *out_dev, const uint64_t *out_offsets_dev, int32_t *status_dev, void *stream,
                                  csgv_decode_tuning *best);

/*
 * Read or set a volume's decode configuration (for instance one found by an
 * earlier autotune).  csgv_decode_set_tuning checks every field against the
 * values listed above (CSGV_ERR_INVALID_ARG otherwise; t->ms is ignored) and
 * applies to decodes issued after it returns.  No counterpart in the paper.
 */
CSGV_API int csgv_decode_get_tuning(const csgv_volume *vol, csgv_decode_tuning *t);
CSGV_API int csgv_decode_set_tuning(csgv_volume *vol, const csgv_decode_tuning *t);

/*
 * Kernel timing (measurement aid; the paper has no counterpart).  While
 * enabled, every kernel the library launches is bracketed by two CUDA events
 * recorded on the launching stream.  csgv_profile_read synchronises the device,
 * sums the elapsed time and launch count per kernel name into the caller's
 * arrays (names: max_kernels entries of 48 bytes, NUL-terminated), sets
 * *n_kernels, and clears the records.  Enabling costs two event records per
 * launch; disabled (the default) it costs nothing.  Returns CSGV_ERR_INVALID_ARG
 * for NULL outputs, CSGV_ERR_CUDA if an event fails.
 *
 * The events come from a per-device pool that csgv_profile_read refills with the
 * events it has read; a launch timed while the pool is empty creates its events,
 * which costs host time between launches.  csgv_profile_reserve adds n_events
 * new events for the current device to the pool, so that a timed run of known
 * length (two events per launch) creates none.  The library owns them until the
 * process ends.  Returns CSGV_ERR_CUDA if an event cannot be created (the events
 * made before it stay in the pool).
 */
CSGV_API int csgv_profile_enable(int on);
CSGV_API int csgv_profile_reserve(uint32_t n_events);
CSGV_API int csgv_profile_read(uint32_t max_kernels, char *names, double *total_ms, uint32_t *launches,
                               uint32_t *n_kernels);

#ifdef __cplusplus
}
#endif
#endif /* CSGV_H */
