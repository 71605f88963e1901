/* Serving engine of the exact packed string matching library (see epsm.h).
 *
 * The paper (Section 1) defines one search: all occurrences of p in t.  This
 * engine has no counterpart in the paper: it keeps texts (corpora) resident
 * in device memory and answers a stream of (corpus, pattern) queries with
 * continuous batching.  Queries that arrive while earlier ones are on the GPU
 * wait in a queue; whenever one of `inflight` launch slots is free, every
 * queued query (up to `max_batch`) goes into one batched launch
 * (epsm_search_batch's kernel: queries on the same corpus share one pass over
 * it), so the work of consecutive batches overlaps on the device.  A batch of
 * at most `small_batch` distinct queries runs as single searches instead, and
 * in a larger batch the queries of m <= 4 on corpora of at least 16 MiB (of
 * m <= 10 when the batch's patterns on that corpus use at most 4 distinct
 * bytes) run as single searches after the batched launch, their positions
 * placed after the batch's in the same output buffer (such queries cost as
 * much in the shared pass as alone, and a single search's pass is cheaper).
 * Texts
 * uploaded at run time are admitted against free device memory and an upload
 * budget, evicting the least recently used idle uploads first; their copies
 * run on a separate stream and overlap the searches.
 *
 * Results are exact: each query's count and sorted positions equal those of
 * epsm_search on the same text, whatever else shares its batch.
 *
 * Threads: the engine runs a scheduler thread and an upload thread.  All
 * functions below may be called from any host thread.
 * Errors: functions return EPSM_ERR_ARG for invalid arguments (unknown or
 * evicted corpus, m outside 1..32, NULL pointers) and EPSM_ERR_CUDA /
 * EPSM_ERR_NOMEM when the device fails; per-request errors are reported in
 * epsm_result.status. */
#ifndef EPSM_SERVE_H
#define EPSM_SERVE_H

#include <stdint.h>

#include "epsm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct epsm_server epsm_server;

typedef struct epsm_server_config {
    uint32_t max_batch;      /* queries per batched launch (0: 1024) */
    uint32_t inflight;       /* launches on the device at once, 1..4 (0: 2) */
    uint32_t per_query;      /* 1: one single-search launch per query instead of batches
                                (the plain per-query path, for comparison) */
    uint32_t small_batch;    /* a batch of at most this many distinct queries runs as
                                single searches, whose fixed cost is lower than a
                                batched launch's (0: 3; at most 8) */
    uint64_t upload_budget;  /* device bytes uploaded texts may hold (0: no budget beyond
                                free memory minus `reserve`) */
    uint64_t reserve;        /* device bytes admission leaves free (0: 4 GiB) */
    uint64_t out_capacity;   /* positions of a fresh output buffer (0: 2^24); buffers grow
                                on demand and are reused */
} epsm_server_config;

typedef struct epsm_result {
    uint64_t request;          /* id returned by submit / upload */
    int32_t status;            /* epsm_status of the request */
    uint32_t corpus;           /* the query's corpus, or the id of an uploaded text */
    uint64_t count;            /* queries: occurrences; uploads: text length */
    const uint64_t *positions; /* queries: DEVICE memory holding `count` sorted start
                                  positions, valid until epsm_server_release */
    int64_t submit_ns;         /* steady-clock time of submission */
    int64_t done_ns;           /* steady-clock time the result was published */
} epsm_result;

/* Creates an engine on `device` (cfg may be NULL for the defaults). */
epsm_status epsm_server_create(epsm_server **out, int device, const epsm_server_config *cfg);

/* Waits for all submitted work, then frees everything the engine owns
 * (uploaded texts, buffers, threads).  Unreleased results become invalid. */
epsm_status epsm_server_destroy(epsm_server *srv);

/* Registers a resident corpus: `text` is DEVICE memory owned by the caller,
 * valid until the engine is destroyed; never evicted. */
epsm_status epsm_server_add_corpus(epsm_server *srv, const uint8_t *text, uint64_t n,
                                   uint32_t *corpus);

/* Uploads a HOST text of n bytes as a new corpus (asynchronous).  The request
 * completes (epsm_result.corpus = the new id) once the text is resident; it
 * waits while admission finds no room.  `text` must stay valid until then. */
epsm_status epsm_server_upload(epsm_server *srv, const uint8_t *text, uint64_t n,
                               uint64_t *request);

/* Queues a query (pattern in HOST memory, copied). */
epsm_status epsm_server_submit(epsm_server *srv, uint32_t corpus, const uint8_t *pattern,
                               uint32_t m, uint64_t *request);

/* Completed requests, oldest first: up to `max` results, waiting at most
 * timeout_ns for the first one.  Returns how many were written. */
uint32_t epsm_server_poll(epsm_server *srv, epsm_result *out, uint32_t max, int64_t timeout_ns);

/* Copies up to `max` positions of a completed, unreleased query to HOST memory. */
epsm_status epsm_server_read(epsm_server *srv, uint64_t request, uint64_t *host, uint64_t max);

/* Ends a query's hold on its output buffer (its positions pointer becomes invalid). */
epsm_status epsm_server_release(epsm_server *srv, uint64_t request);

/* Load replay for measurement: submits items[i] at start + at_ns (a query on
 * `corpus` with pattern data[0..len), or, if kind == 1, an upload of the host
 * text data[0..len)), collects every result, releases it, and reports per
 * item the latency (publication - scheduled arrival), the count and the
 * status, and the time from start to the last result.  Not to be mixed with
 * other submissions on the same engine. */
typedef struct epsm_replay_item {
    int64_t at_ns;
    uint32_t kind;           /* 0: query, 1: upload */
    uint32_t corpus;
    const uint8_t *data;
    uint64_t len;
} epsm_replay_item;

epsm_status epsm_server_replay(epsm_server *srv, uint32_t nitems, const epsm_replay_item *items,
                               int64_t *latency_ns, uint64_t *counts, int32_t *status,
                               int64_t *elapsed_ns);

/* Engine counters: batches launched, queries served, uploads admitted, texts
 * evicted, output-buffer regrowths (a batch re-run after an overflow). */
typedef struct epsm_server_stats {
    uint64_t batches;
    uint64_t queries;
    uint64_t uploads;
    uint64_t evictions;
    uint64_t reruns;
    uint64_t max_batch_seen;
} epsm_server_stats;

epsm_status epsm_server_stats_get(epsm_server *srv, epsm_server_stats *out);

/* Host-side fault injection (for testing the engine's failure handling; no
 * GPU fault is involved).  Arms `count` more failures of one kind, each of
 * which fires once, at the next point of that kind:
 *   EPSM_FAULT_ALLOC   obtaining an output buffer for a batch fails: every
 *                      query of that batch completes with EPSM_ERR_NOMEM;
 *   EPSM_FAULT_ADMIT   admission refuses an upload: the upload completes with
 *                      EPSM_ERR_NOMEM;
 *   EPSM_FAULT_UPLOAD  an upload's copy to the device fails: the upload
 *                      completes with EPSM_ERR_CUDA and its memory is freed.
 * The engine keeps serving afterwards.  The environment variable EPSM_FAULT,
 * read when an engine is created, arms the same (e.g. "alloc:2,upload:1").
 * EPSM_ERR_ARG for a NULL engine or an unknown kind. */
#define EPSM_FAULT_ALLOC 0
#define EPSM_FAULT_ADMIT 1
#define EPSM_FAULT_UPLOAD 2
epsm_status epsm_server_inject_fault(epsm_server *srv, int kind, uint32_t count);

#ifdef __cplusplus
}
#endif

#endif /* EPSM_SERVE_H */
