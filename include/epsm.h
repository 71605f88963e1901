/*
 * epsm.h — C ABI of the GB300 exact short-pattern matching library.
 *
 * Operation (Section 1 and Section 2 of Faro & Kulekci, "Fast Packed String
 * Matching for Short Patterns"): given a text t[0..n-1] and a pattern
 * p[0..m-1] of bytes, report ALL start positions s with 0 <= s <= n-m and
 * t[s+i] == p[i] for every i < m.  Overlapping occurrences are all reported,
 * bytes compare as unsigned values, and positions are 0-based uint64 in
 * ascending order.  The library implements the three length regimes of
 * Section 3 (a packed window compare for very short patterns, a first-bytes
 * filter plus in-register verify for short patterns, an aligned-block
 * fingerprint filter plus verify for medium patterns) as sm_103a kernels.
 *
 * Conventions for every entry point:
 *   - 1 <= m <= EPSM_MAX_M (32); m == 0 or m > 32 returns EPSM_ERR_ARG, except
 *     that the single-search entry points (epsm_search, epsm_search_async,
 *     epsm_search_variant with EPSM_VARIANT_AUTO or EPSM_VARIANT_BLOCK8) take
 *     m up to EPSM_MAX_M_LONG (4096).
 *   - m > n is not an error: the count is 0.
 *   - Inputs are never modified.  Buffers named "device" must be device
 *     memory of the context's device (or managed memory); buffers named "host"
 *     are ordinary host memory (pinned memory makes copies faster).
 *   - If the number of occurrences exceeds `capacity`, the first `capacity`
 *     positions are written, the true count is reported, and the call returns
 *     EPSM_ERR_CAPACITY.  capacity == 0 (positions may then be NULL) counts
 *     only.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL is the CUDA default
 *     stream).  A context is not thread-safe: use one context per host
 *     thread.  Calls on one context that use different streams are ordered
 *     by the context (each call waits for the previous one's scratch use).
 *   - A bounded device-side wait that gives up makes the call return
 *     EPSM_ERR_TIMEOUT; the context stays usable.
 *   - The library allocates device scratch inside the context only (tile
 *     status words, counters, staging buffers); it never frees caller memory.
 */
#ifndef EPSM_H
#define EPSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EPSM_MAX_M 32u
/* Longest pattern of the single-search entry points (epsm_search,
 * epsm_search_async, epsm_search_variant): m > EPSM_MAX_M uses the 8-byte
 * block variant on the first 32 bytes and checks the rest at each candidate. */
#define EPSM_MAX_M_LONG 4096u

typedef struct epsm_ctx epsm_ctx;

typedef enum {
    EPSM_OK = 0,
    EPSM_ERR_ARG = 1,       /* bad argument (NULL pointer, m out of range, ...) */
    EPSM_ERR_CAPACITY = 2,  /* more occurrences than capacity; true count reported */
    EPSM_ERR_CUDA = 3,      /* a CUDA runtime call failed */
    EPSM_ERR_NOMEM = 4,     /* scratch or staging allocation failed */
    EPSM_ERR_TIMEOUT = 5    /* a bounded device wait gave up; results are invalid */
} epsm_status;

/* Search variants (the length regimes of Section 3 mapped to GPU kernels).
 * EPSM_VARIANT_AUTO lets the context's tuning table choose by m. */
typedef enum {
    EPSM_VARIANT_AUTO = 0,
    EPSM_VARIANT_DIRECT = 1,   /* packed window compare, 1 <= m <= 4   (Section 3.2, EPSMa) */
    EPSM_VARIANT_PREFIX4 = 2,  /* 4-byte first-bytes filter + verify, 4 <= m <= 15 (Section 3.3, EPSMb) */
    EPSM_VARIANT_PREFIX8 = 3,  /* 8-byte first-bytes filter + verify, 8 <= m <= 15 (Section 3.3, EPSMb with m' = 8) */
    EPSM_VARIANT_BLOCK8 = 4,   /* aligned 8-byte block fingerprint + verify, 15 <= m <= 32 (Section 3.4, EPSMc) */
    EPSM_VARIANT_BLOCK4 = 5,   /* aligned 4-byte blocks compared with the pattern's 4 blocks + verify,
                                  7 <= m <= 16 (Section 3.4's aligned-block idea with 4-byte blocks) */
    EPSM_VARIANT_CODE2 = 6,    /* 2-bit codes (bits 1..2 of every byte) of the first min(m, 8) bytes
                                  as the filter + verify, 2 <= m <= 16 (Section 3.3's filter-then-verify) */
    EPSM_VARIANT_ADAPT = 7,    /* 5 <= m <= 16: per block, the 2-bit code filter where the text makes
                                  4-byte block matches frequent (small alphabets), else BLOCK4
                                  (m >= 7) or PREFIX4 */
    EPSM_VARIANT_BLOCK8S = 8   /* 23 <= m <= 32, single search: BLOCK8 with the block stride sh of
                                  Section 3.4 (every second aligned block inspected, 16 pattern blocks
                                  in the table); batched searches run it as BLOCK8 */
} epsm_variant;

/* Create a context on CUDA device `device`.  `flags` is reserved (pass 0).
 * On success *out owns a stream and lazily grown device scratch. */
epsm_status epsm_create(epsm_ctx **out, int device, uint64_t flags);

/* Release the context, its stream and its scratch.  NULL is accepted. */
epsm_status epsm_destroy(epsm_ctx *ctx);

/* Human-readable name of a status code (static storage). */
const char *epsm_status_str(epsm_status s);

/* Last CUDA error string seen by the context (static or context storage). */
const char *epsm_last_error(epsm_ctx *ctx);

/* Single search, synchronous (Section 1 problem; Section 3 procedures).
 *   text      device, n bytes (any alignment), caller-owned
 *   pattern   host, m bytes, copied before the call returns
 *   positions device, room for `capacity` uint64, caller-owned (NULL iff capacity == 0)
 *   count     host: receives the true number of occurrences
 * Returns after the result is complete. */
epsm_status epsm_search(epsm_ctx *ctx, const uint8_t *text, uint64_t n,
                        const uint8_t *pattern, uint32_t m,
                        uint64_t *positions, uint64_t capacity,
                        uint64_t *count, void *stream);

/* Single search, asynchronous: like epsm_search, but `count_dev` is DEVICE
 * memory that receives the true count when the enqueued work completes, and the
 * call returns once the work is enqueued.  Capacity overflow and device wait
 * timeouts are reported by the next epsm_sync on the context. */
epsm_status epsm_search_async(epsm_ctx *ctx, const uint8_t *text, uint64_t n,
                              const uint8_t *pattern, uint32_t m,
                              uint64_t *positions, uint64_t capacity,
                              uint64_t *count_dev, void *stream);

/* Same as epsm_search_async with an explicit variant (EPSM_VARIANT_AUTO picks
 * by the tuning table).  A variant that does not cover m returns EPSM_ERR_ARG. */
epsm_status epsm_search_variant(epsm_ctx *ctx, int variant, const uint8_t *text, uint64_t n,
                                const uint8_t *pattern, uint32_t m,
                                uint64_t *positions, uint64_t capacity,
                                uint64_t *count_dev, void *stream);

/* Wait for the context's outstanding work on `stream` (NULL = default stream)
 * and report device-side errors raised since the last sync: EPSM_ERR_TIMEOUT
 * if a bounded wait gave up, EPSM_ERR_CAPACITY if an asynchronous search found
 * more occurrences than its capacity, EPSM_ERR_CUDA on a CUDA error. */
epsm_status epsm_sync(epsm_ctx *ctx, void *stream);

/* Diagnostic of the bounded device waits: launches one warp that waits for a
 * device flag nothing sets, giving up after limit_ns (1 ns .. 1 s) exactly as
 * the search kernels' waits do.  The next epsm_sync returns EPSM_ERR_TIMEOUT
 * and clears the condition; the context stays usable.  EPSM_ERR_ARG for a
 * NULL context or a limit outside that range. */
epsm_status epsm_wait_probe(epsm_ctx *ctx, uint64_t limit_ns, void *stream);

/* Batched search over `npairs` independent (text, pattern) pairs of uneven n
 * and m, in one persistent launch (each pair is one Section 1 problem).
 *   texts      host array of npairs DEVICE text pointers
 *   ns         host array of npairs text lengths
 *   patterns   host array of npairs HOST pattern pointers
 *   ms         host array of npairs pattern lengths (each 1..32)
 *   positions  device pool of `capacity` uint64; pair i's sorted positions are
 *              written at [offsets[i], offsets[i+1])
 *   offsets    host array of npairs+1 entries (offsets[npairs] = total count)
 * Synchronous.  Pool overflow returns EPSM_ERR_CAPACITY with offsets filled. */
epsm_status epsm_search_batch(epsm_ctx *ctx, uint32_t npairs,
                              const uint8_t *const *texts, const uint64_t *ns,
                              const uint8_t *const *patterns, const uint32_t *ms,
                              uint64_t *positions, uint64_t capacity,
                              uint64_t *offsets, void *stream);

/* End-to-end search from HOST memory: copies the text to the device, runs one
 * single search (the kernels of epsm_search, automatic variant) per pattern
 * on it, and copies the positions back.
 *   text_host      host, n bytes
 *   patterns_host  host, concatenation of the npat patterns
 *   ms             host, npat pattern lengths (each 1..EPSM_MAX_M_LONG)
 *   positions_host host, room for `capacity` uint64 (pinned memory makes the
 *                  copy faster)
 *   offsets_host   host, npat+1 entries (pattern k's positions are at
 *                  [offsets[k], offsets[k+1]); offsets[npat] = total)
 * Synchronous.  Device staging for the text and `capacity` positions lives in
 * the context (grown on demand).  If the total exceeds `capacity`, the first
 * `capacity` positions are copied, the offsets are the true ones, and the call
 * returns EPSM_ERR_CAPACITY. */
/* Variant the context uses for pattern length m under EPSM_VARIANT_AUTO on the
 * longest texts (the last bucket of the tuning table below). */
int epsm_variant_for(epsm_ctx *ctx, uint32_t m);

/* Override the automatic variant for pattern length m (1..32) in every bucket
 * of the tuning table; `variant` must cover m. */
epsm_status epsm_set_variant(epsm_ctx *ctx, uint32_t m, int variant);

/* Tuning table of a context.  For each text-length bucket and pattern length
 * m (1..32; longer patterns use the m = 32 entry's shape and width) the table
 * holds:
 *   variant  the kernel variant EPSM_VARIANT_AUTO picks (must cover m);
 *   shape    the filter kernel's launch shape: 0 = a 6-stage ring of 16 KiB
 *            stages with 2 blocks per SM, 1 = a 4-stage ring with 3 blocks per
 *            SM (the default);
 *   kbits    the width k of the block variants' fingerprint table, 2^k bits
 *            (Section 3.4 takes k = 11; default 14; EPSM_KBITS_MIN..MAX).
 * Buckets: n < EPSM_BUCKET1_MIN, n < EPSM_BUCKET2_MIN, and larger texts.
 * The results do not depend on the table, only the speed does. */
#define EPSM_TEXT_BUCKETS 3
#define EPSM_BUCKET1_MIN (16ull << 20)
#define EPSM_BUCKET2_MIN (512ull << 20)
#define EPSM_KBITS_MIN 8u
#define EPSM_KBITS_MAX 14u

/* Sets the entry of one bucket (0..2) or of all buckets (bucket = -1) for m:
 * variant EPSM_VARIANT_AUTO, shape -1 or kbits 0 keep the current value.
 * EPSM_ERR_ARG for a value out of range or a variant that does not cover m. */
epsm_status epsm_set_tuning(epsm_ctx *ctx, int bucket, uint32_t m, int variant, int shape,
                            uint32_t kbits);

/* Reads the entry of bucket (0..2) for m; NULL outputs are skipped. */
epsm_status epsm_get_tuning(epsm_ctx *ctx, int bucket, uint32_t m, int *variant, int *shape,
                            uint32_t *kbits);

/* Number of kernel launches the context has issued (all entry points). */
uint64_t epsm_launch_count(epsm_ctx *ctx);

/* 1 if the context's batched submissions replay a captured CUDA graph
 * (upload, pattern-table build, batched scan, offsets download), 0 if they are
 * launched directly (no batch run yet, or graph capture unavailable). */
int epsm_batch_uses_graph(epsm_ctx *ctx);

/* Largest text epsm_search_static accepts (bytes). */
#define EPSM_STATIC_MAX_TEXT (64ull << 20)

/* Single search that allocates nothing and needs no context.
 *
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory themselves (a framework that routes every
 * allocation through its own pool, a real-time loop where an allocation could
 * stall or fail, a plug-in whose host pre-sizes all memory).  The search runs
 * the kernels of epsm_search_async with the library's built-in per-m variant
 * choice (a context may have installed a measured table instead; the positions
 * are the same, the speed can differ); its scratch lives in a fixed device
 * array of about 8.5 MiB inside the library, which every GPU that loads the
 * library keeps until the process exits.
 *   text        device, n bytes, n <= EPSM_STATIC_MAX_TEXT (larger n returns
 *               EPSM_ERR_ARG without touching the GPU)
 *   pattern     host, m bytes (1..32)
 *   positions   device, room for `capacity` uint64 (NULL iff capacity == 0)
 *   result_dev  device, two uint64: [0] receives the count, [1] the device
 *               error bits (1: a bounded wait gave up, 2: more occurrences than
 *               capacity); both are cleared when the call is enqueued
 * Asynchronous on `stream` (NULL = default stream) on the current device.
 * The first call on a device looks up the array's device address and the SM
 * count and clears the array's counters, waiting on `stream` for the clearing
 * to complete; make that first call before any stream capture.  Calls share
 * the one array: calls whose work overlaps on the GPU (different streams, or
 * another host thread) race and give wrong results; order them on one stream.
 * It calls no cudaMalloc, cudaFree or other allocating routine. */
epsm_status epsm_search_static(const uint8_t *text, uint64_t n, const uint8_t *pattern,
                               uint32_t m, uint64_t *positions, uint64_t capacity,
                               uint64_t *result_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* EPSM_H */
