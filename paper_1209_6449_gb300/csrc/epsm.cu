// Host runtime and C ABI of the exact short-pattern matching library (see
// include/epsm.h for the contract of every entry point).
//
// The runtime validates arguments, picks the kernel variant for the pattern
// length (Section 3: the EPSM dispatcher chooses its procedure by m), packs
// the pattern, sizes the persistent grid from the SM count and the kernel's
// occupancy, manages the context's device scratch (look-back status words,
// tile ticket, error word) and enqueues the kernels.  Every step of the
// search itself runs in the kernels of epsm_kernels.cuh.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "epsm.h"
#include "epsm_kernels.cuh"
#include "epsm_stream.cuh"
#include "epsm_group.cuh"

using namespace epsm;

namespace {
constexpr uint32_t kMaxRanges = 16384;  // range-total scratch of a context (emit ranges)
constexpr int kMaxDevices = 64;         // devices the per-device caches below cover

// Resident blocks per SM of `kernel` on the CURRENT device, worked out once
// per device: the dynamic shared-memory opt-in (cudaFuncSetAttribute) belongs
// to a device's context, so a second device needs its own set-up.  `cache`
// holds one entry per device (0: not yet known); concurrent first calls on a
// device may both do the set-up, which is harmless.  Returns 0 on a CUDA
// error or a device index beyond the cache.
template <typename K>
int blocks_per_sm(K kernel, int threads, size_t smem, int cap, std::atomic<int> (&cache)[kMaxDevices]) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
    const int known = cache[dev].load(std::memory_order_acquire);
    if (known > 0) return known;
    if (smem > 0 && cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem) != cudaSuccess)
        return 0;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess) return 0;
    const int v = std::max(1, cap > 0 ? std::min(b, cap) : b);
    cache[dev].store(v, std::memory_order_release);
    return v;
}

// Makes a context's device current for the duration of a call and restores
// the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; prev = -1; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};
}

#define EPSM_API extern "C" __attribute__((visibility("default")))

namespace {

// Built-in per-m choice (a context may install a measured table instead):
// the packed compare for m <= 4, the adaptive 4-byte block / 2-bit code filter
// up to 16, the 8-byte block fingerprint above, with the block stride for
// m >= 23.
int default_variant(uint32_t m) {
    if (m <= 4) return V_DIRECT;
    if (m <= 16) return V_ADAPT;
    if (m <= 22) return V_BLOCK8;
    return V_BLOCK8S;
}

bool variant_covers(int v, uint32_t m) {
    switch (v) {
        case V_DIRECT: return m >= 1 && m <= 4;
        case V_PREFIX4: return m >= 4 && m <= 15;
        case V_PREFIX8: return m >= 8 && m <= 15;
        case V_BLOCK8: return m >= 15 && m <= 32;
        case V_BLOCK4: return m >= 7 && m <= 16;
        case V_CODE2: return m >= 2 && m <= 16;
        case V_ADAPT: return m >= 5 && m <= 16;
        case V_BLOCK8S: return m >= 23 && m <= 32;
        default: return false;
    }
}

int variant_offset(int v) { return v == V_BLOCK8 ? -7 : v == V_BLOCK8S ? -15 : 0; }

Pattern pack_pattern(const uint8_t *p, uint32_t m) {
    Pattern pat;
    memset(&pat, 0, sizeof(pat));
    uint8_t bytes[32];
    memset(bytes, 0, sizeof(bytes));
    memcpy(bytes, p, m);
    for (int i = 0; i < 8; ++i)
        pat.w[i] = (uint32_t)bytes[4 * i] | ((uint32_t)bytes[4 * i + 1] << 8) |
                   ((uint32_t)bytes[4 * i + 2] << 16) | ((uint32_t)bytes[4 * i + 3] << 24);
    pat.m = m;
    pat.kbits = kHashBitsDefault;
    // smallest period up to 8 (the block variants' run shortcut), and the
    // last 8 bytes
    pat.q = 0;
    for (uint32_t q = 1; q <= 8 && q < m; ++q) {
        uint32_t i = 0;
        while (i + q < m && p[i] == p[i + q]) ++i;
        if (i + q == m) { pat.q = q; break; }
    }
    if (m >= 8) {
        uint8_t t8[8];
        memcpy(t8, p + m - 8, 8);
        pat.tl = (uint32_t)t8[0] | ((uint32_t)t8[1] << 8) | ((uint32_t)t8[2] << 16) | ((uint32_t)t8[3] << 24);
        pat.th = (uint32_t)t8[4] | ((uint32_t)t8[5] << 8) | ((uint32_t)t8[6] << 16) | ((uint32_t)t8[7] << 24);
    }
    return pat;
}

SearchJob make_job(const uint8_t *text, uint64_t n, const Pattern &pat) {
    SearchJob J;
    uintptr_t t = reinterpret_cast<uintptr_t>(text);
    J.base = reinterpret_cast<const uint8_t *>(t & ~(uintptr_t)15);
    J.delta = (uint64_t)(t & 15);
    J.lim = J.delta + n;
    J.pmax = (int64_t)(J.delta + n) - (int64_t)pat.m;
    J.pat = pat;
    return J;
}

// Per-context resources of the batched launch: one pinned staging buffer
// holding the header and the job table, device copies of both, the
// fingerprint tables, the job offsets, and the CUDA graph of the submission
// (header/jobs upload -> table build -> batched scan -> offsets download),
// built once per capacity and replayed for every batch that fits.
struct BatchRes {
    uint8_t *hstage = nullptr;  // pinned: Header | JobDesc[] | GroupDesc[] | uint32 group_jobs[]
    uint8_t *dstage = nullptr;
    uint64_t *hoff = nullptr;   // pinned: job offsets + total
    uint64_t *doff = nullptr;
    uint8_t *tables = nullptr;  // cap block-variant tables
    uint8_t *comb = nullptr;    // comb_cap shared tables
    unsigned long long *rt = nullptr;  // per-range hit totals of the batched launch
    uint32_t cap = 0;           // jobs (and groups)
    uint32_t comb_cap = 0;
    cudaGraph_t graph = nullptr;     // kept: its node handles address the exec's copies
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t up = nullptr, down = nullptr;
    uint32_t *seg_count = nullptr;   // per pattern segment: hits
    uint32_t *seg_off = nullptr;     // per pattern segment: hit list in pool
    uint64_t seg_cap = 0;
    uint16_t *pool = nullptr;        // hit lists
    uint64_t pool_alloc = 0;
    uint32_t *pool_ctr = nullptr;
    // the submitted batch, for batch_complete
    std::vector<int32_t> pend_jidx;  // pair -> job (-1: no stages)
    uint32_t pend_npairs = 0;
    uint32_t pend_nj = 0;
    uint64_t pend_capacity = 0;
    uint64_t gen = 1;                // bumped when a buffer the graph uses moves
    uint64_t graph_gen = 0;          // generation the graph was built with
    bool graph_failed = false;       // a build failed once: launch directly
    int grid = 0;   // filter kernel blocks
    int egrid = 0;  // emission kernel blocks
};

constexpr size_t kBatchHdrBytes = 128;  // Header, padded to keep JobDesc aligned

size_t batch_jobs_off() { return kBatchHdrBytes; }
size_t align16(size_t x) { return (x + 15u) & ~(size_t)15u; }
// Staging: Header | JobDesc[nj] | GroupDesc[ng] | uint32 group_jobs[nj], each
// part 16-byte aligned, packed after the jobs actually used (the upload is
// only as large as the batch); sized for cap jobs and cap groups.
size_t batch_stage_bytes(uint32_t cap) {
    return kBatchHdrBytes + align16((size_t)cap * sizeof(group::JobDesc)) +
           align16((size_t)cap * sizeof(group::GroupDesc)) + (size_t)cap * sizeof(uint32_t);
}

}  // namespace

struct Tune {
    int variant;
    int shape;
    uint32_t kbits;
};

// Text-length bucket of the tuning table (boundaries in include/epsm.h).
int text_bucket(uint64_t n) {
    return n < EPSM_BUCKET1_MIN ? 0 : n < EPSM_BUCKET2_MIN ? 1 : 2;
}

struct epsm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sms = 0;
    DevMisc *misc = nullptr;     // device
    DevMisc *hmisc = nullptr;    // pinned host mirror
    cudaEvent_t ev = nullptr;
    cudaStream_t last_stream = nullptr;
    bool have_ev = false;
    // tuning table: per text-length bucket and pattern length, the variant,
    // the filter kernel's launch shape and the block fingerprint width
    Tune tune[EPSM_TEXT_BUCKETS][EPSM_MAX_M + 1];
    uint64_t launches = 0;
    char errbuf[256];
    // batched launch
    BatchRes batch;
    // streaming-kernel scratch
    uint32_t *seg_count = nullptr;
    uint16_t *seg_mask = nullptr;
    unsigned long long *range_total = nullptr;
    uint64_t seg_cap = 0;
    // host end-to-end staging
    uint8_t *dtext = nullptr;
    uint64_t dtext_cap = 0;
    uint64_t *dpos = nullptr;
    uint64_t dpos_cap = 0;
    // pattern bytes past the first 32 of a long pattern (m > EPSM_MAX_M)
    uint8_t *tail = nullptr;
    uint32_t tail_cap = 0;
    // host end-to-end: copies of finished patterns' positions overlap the
    // next pattern's search
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_ev = nullptr;
};

namespace {

epsm_status cuda_fail(epsm_ctx *c, cudaError_t e, const char *what) {
    if (c) snprintf(c->errbuf, sizeof(c->errbuf), "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? EPSM_ERR_NOMEM : EPSM_ERR_CUDA;
}

#define CK(call)                                               \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

// NULL is the CUDA default stream, as for every CUDA library call.
cudaStream_t pick_stream(epsm_ctx *c, void *s) {
    (void)c;
    return (cudaStream_t)s;
}

// Orders this call after the previous call of the context when it used
// another stream (the scratch words are shared).
epsm_status order_after_previous(epsm_ctx *c, cudaStream_t s) {
    if (c->have_ev && c->last_stream != s) CK(cudaStreamWaitEvent(s, c->ev, 0));
    return EPSM_OK;
}

epsm_status mark_done(epsm_ctx *c, cudaStream_t s) {
    CK(cudaEventRecord(c->ev, s));
    c->have_ev = true;
    c->last_stream = s;
    return EPSM_OK;
}


// Scratch of the streaming kernel: one count per 2 KiB segment and 128 chunk
// masks (256 B) per segment, i.e. n/512 + n/8 bytes; status words for the blocks.
epsm_status ensure_stream_scratch(epsm_ctx *c, uint64_t nstages, cudaStream_t s) {
    if (!c->range_total) {
        CK(cudaMalloc(&c->range_total, kMaxRanges * sizeof(unsigned long long)));
        CK(cudaMemsetAsync(c->range_total, 0, kMaxRanges * sizeof(unsigned long long), s));
    }
    const uint64_t nseg = nstages * stream::kConsumerWarps;
    if (nseg <= c->seg_cap) return EPSM_OK;
    uint64_t cap = std::max<uint64_t>(nseg, c->seg_cap * 2);
    CK(cudaStreamSynchronize(s));
    if (c->seg_count) CK(cudaFree(c->seg_count));
    if (c->seg_mask) CK(cudaFree(c->seg_mask));
    c->seg_count = nullptr;
    c->seg_mask = nullptr;
    c->seg_cap = 0;
    CK(cudaMalloc(&c->seg_count, cap * sizeof(uint32_t)));
    CK(cudaMalloc(&c->seg_mask, cap * stream::kSegChunks * sizeof(uint16_t)));
    c->seg_cap = cap;
    return EPSM_OK;
}


// Emit ranges of a single search: when positions are wanted, many (claimed
// dynamically by the emission kernel), each at least one batch of 256
// segments (32 stages); for a count only, a single one.

int stream_emit_grid(int sms) {
    static std::atomic<int> cache[kMaxDevices];
    return sms * blocks_per_sm(stream_emit_kernel, stream::kEmitThreads, 0, 0, cache);
}

// A single search: the streaming filter kernel (epsm_stream.cuh; up to two
// blocks per SM), then, when positions are wanted, the emission kernel.
template <int V, int MP, int SH>
cudaError_t launch_stream_t(int sms, stream::StreamParams &p, cudaStream_t s) {
    static std::atomic<int> cache[kMaxDevices];
    const size_t smem = sizeof(stream::StreamSmem<stream::Shape<SH>::stages>);
    const int per_sm = blocks_per_sm(stream_kernel<V, MP, SH>, stream::kThreadsStream, smem,
                                     stream::Shape<SH>::blocks, cache);
    if (per_sm == 0) return cudaErrorInvalidDevice;
    uint64_t grid = std::min<uint64_t>(std::max<uint64_t>(p.nstages, 1u), (uint64_t)sms * per_sm);
    grid = std::min<uint64_t>(grid, stream::kMaxBlocks);
    const uint64_t nst = std::max<uint64_t>(p.nstages, 1u);
    // count only: one range, which every filter warp adds its total to once
    const uint64_t want = p.emit ? std::max<uint64_t>(1, std::min<uint64_t>(nst / 32u, kMaxRanges)) : 1u;
    p.range_stages = (nst + want - 1) / want;
    p.nranges = (uint32_t)((nst + p.range_stages - 1) / p.range_stages);
    p.off = variant_offset(V);
    // both kernels are launched as programmatic dependents of the previous
    // kernel of the stream: each waits on the device (grid_dep_wait) for its
    // predecessor to finish, so their launch latency overlaps the predecessor
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(stream::kThreadsStream);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, stream_kernel<V, MP, SH>, p);
    if (e != cudaSuccess || !p.emit) return e;
    const int eg = stream_emit_grid(sms);
    if (eg == 0) return cudaErrorUnknown;
    cfg.gridDim = dim3((unsigned)eg);
    cfg.blockDim = dim3(stream::kEmitThreads);
    cfg.dynamicSmemBytes = 0;
    return cudaLaunchKernelEx(&cfg, stream_emit_kernel, p);
}

template <int SH>
cudaError_t launch_stream_shape(int sms, int v, uint32_t m, stream::StreamParams &p, cudaStream_t s) {
    switch (v) {
        case V_DIRECT:
            switch (m) {
                case 1: return launch_stream_t<V_DIRECT, 1, SH>(sms, p, s);
                case 2: return launch_stream_t<V_DIRECT, 2, SH>(sms, p, s);
                case 3: return launch_stream_t<V_DIRECT, 3, SH>(sms, p, s);
                default: return launch_stream_t<V_DIRECT, 4, SH>(sms, p, s);
            }
        case V_PREFIX4: return launch_stream_t<V_PREFIX4, 4, SH>(sms, p, s);
        case V_PREFIX8: return launch_stream_t<V_PREFIX8, 8, SH>(sms, p, s);
        case V_BLOCK4: return launch_stream_t<V_BLOCK4, 4, SH>(sms, p, s);
        case V_CODE2:  // (a pattern of period 1 has a kernel of its own)
            return p.job.pat.q == 1u ? launch_stream_t<V_CODE2, kMpRun, SH>(sms, p, s)
                                     : launch_stream_t<V_CODE2, 4, SH>(sms, p, s);
        case V_ADAPT: return launch_stream_t<V_ADAPT, 4, SH>(sms, p, s);
        case V_BLOCK8S:  // (a pattern of period 1 has a kernel of its own)
            return p.job.pat.q == 1u && p.job.pat.m <= 32u ? launch_stream_t<V_BLOCK8S, kMpRun, SH>(sms, p, s)
                                                           : launch_stream_t<V_BLOCK8S, 8, SH>(sms, p, s);
        default: return launch_stream_t<V_BLOCK8, 8, SH>(sms, p, s);
    }
}

// A single search with the filter kernel's launch shape `shape` (0: 6-stage
// ring, 2 blocks per SM; 1: 4-stage ring, 3 blocks per SM).
cudaError_t launch_stream(int sms, int v, uint32_t m, int shape, stream::StreamParams &p,
                          cudaStream_t s) {
    return shape == 0 ? launch_stream_shape<0>(sms, v, m, p, s) : launch_stream_shape<1>(sms, v, m, p, s);
}

// Stages of 16 KiB needed for a job: stage k covers starts [16K*k + OFF, 16K*(k+1) + OFF).
uint64_t stages_for(uint64_t delta, uint64_t n, uint32_t m, int v) {
    if (n < m || n == 0) return 0;
    int64_t pmax = (int64_t)(delta + n - m);
    return (uint64_t)((pmax - variant_offset(v)) / (int64_t)stream::kStageBytes) + 1u;
}

epsm_status search_async_impl(epsm_ctx *c, int variant, const uint8_t *text, uint64_t n,
                              const uint8_t *pattern, uint32_t m, uint64_t *positions,
                              uint64_t capacity, uint64_t *count_dev, void *stream,
                              uint64_t *cursor) {
    if (!c || !pattern || !count_dev) return EPSM_ERR_ARG;
    if (m == 0 || m > EPSM_MAX_M_LONG) return EPSM_ERR_ARG;
    if (n > 0 && !text) return EPSM_ERR_ARG;
    if (capacity > 0 && !positions) return EPSM_ERR_ARG;
    // a long pattern: the 8-byte block filter and check on its first 32
    // bytes, then the rest of the pattern checked at each candidate
    const bool longp = m > EPSM_MAX_M;
    const Tune &T = c->tune[text_bucket(n)][longp ? EPSM_MAX_M : m];
    int v = variant == EPSM_VARIANT_AUTO ? (longp ? V_BLOCK8 : T.variant) : variant;
    if (!(longp ? v == V_BLOCK8 : variant_covers(v, m))) return EPSM_ERR_ARG;
    cudaStream_t s = pick_stream(c, stream);
    epsm_status st = order_after_previous(c, s);
    if (st != EPSM_OK) return st;
    if (n < m) {
        CK(cudaMemsetAsync(count_dev, 0, sizeof(uint64_t), s));
        return mark_done(c, s);
    }
    stream::StreamParams p;
    memset(&p, 0, sizeof(p));
    p.job = make_job(text, n, pack_pattern(pattern, longp ? EPSM_MAX_M : m));
    p.job.pat.kbits = T.kbits;
    if (longp) {
        p.job.pmax = (int64_t)(p.job.delta + n) - (int64_t)m;
        p.job.pat.q = 0;  // (the period shortcut covers patterns of at most 32 bytes)
        const uint32_t mt = m - EPSM_MAX_M;
        if (mt > c->tail_cap) {
            CK(cudaStreamSynchronize(s));
            if (c->tail) CK(cudaFree(c->tail));
            c->tail = nullptr;
            c->tail_cap = 0;
            CK(cudaMalloc(&c->tail, EPSM_MAX_M_LONG));
            c->tail_cap = EPSM_MAX_M_LONG;
        }
        // from pageable host memory: the source is consumed before the call returns
        CK(cudaMemcpyAsync(c->tail, pattern + EPSM_MAX_M, mt, cudaMemcpyHostToDevice, s));
        p.tail = c->tail;
        p.mtail = mt;
    }
    p.nstages = stages_for(p.job.delta, n, m, v);
    p.chunk_full0 = (p.job.delta + 15u) / 16u;
    p.chunk_full1 = p.job.lim / 16u;
    p.emit = capacity > 0 ? 1 : 0;
    p.cursor = cursor;
    if ((st = ensure_stream_scratch(c, p.nstages, s)) != EPSM_OK) return st;
    p.positions = positions;
    p.capacity = capacity;
    p.count_out = count_dev;
    p.seg_count = c->seg_count;
    p.seg_mask = c->seg_mask;
    p.range_total = c->range_total;
    p.err = &c->misc->err;
    p.misc = c->misc;
    CK(launch_stream(c->sms, v, m, T.shape, p, s));
    c->launches += p.emit ? 2 : 1;  // filter kernel (+ emission kernel)
    return mark_done(c, s);
}

// Reads the device scratch words after the stream drained; clears the error word.
epsm_status read_misc(epsm_ctx *c, cudaStream_t s, uint32_t *err) {
    CK(cudaMemcpyAsync(c->hmisc, c->misc, sizeof(DevMisc), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *err = c->hmisc->err;
    if (*err) {
        CK(cudaMemsetAsync(&c->misc->err, 0, sizeof(uint32_t), s));
        CK(cudaStreamSynchronize(s));
    }
    return EPSM_OK;
}


void free_batch(BatchRes &R) {
    if (R.exec) cudaGraphExecDestroy(R.exec);
    if (R.graph) cudaGraphDestroy(R.graph);
    if (R.hstage) cudaFreeHost(R.hstage);
    if (R.dstage) cudaFree(R.dstage);
    if (R.hoff) cudaFreeHost(R.hoff);
    if (R.doff) cudaFree(R.doff);
    if (R.tables) cudaFree(R.tables);
    if (R.comb) cudaFree(R.comb);
    if (R.rt) cudaFree(R.rt);
    if (R.seg_count) cudaFree(R.seg_count);
    if (R.seg_off) cudaFree(R.seg_off);
    if (R.pool) cudaFree(R.pool);
    if (R.pool_ctr) cudaFree(R.pool_ctr);
    R = BatchRes();
}

int batch_grid(int sms) {
    static std::atomic<int> cache[kMaxDevices];
    const int per_sm = blocks_per_sm(group_kernel, stream::kThreadsStream, sizeof(group::Smem),
                                     group::kGroupBlocksPerSm, cache);
    return (int)std::min<uint64_t>((uint64_t)sms * per_sm, stream::kMaxBlocks);
}

// Blocks of the emission kernel: as many as fit (it is latency bound).
int emit_grid(int sms) {
    static std::atomic<int> cache[kMaxDevices];
    return sms * blocks_per_sm(group_emit_kernel, stream::kEmitThreads, 0, 0, cache);
}

void drop_graph(BatchRes &R) {
    if (R.exec) cudaGraphExecDestroy(R.exec);
    if (R.graph) cudaGraphDestroy(R.graph);
    R.exec = nullptr;
    R.graph = nullptr;
}

epsm_status ensure_batch(epsm_ctx *c, uint32_t njobs, uint32_t ncomb, cudaStream_t s) {
    BatchRes &R = c->batch;
    if (!R.hstage || njobs > R.cap) {
        const uint32_t cap = std::max<uint32_t>({njobs, R.cap * 2u, 64u});
        CK(cudaStreamSynchronize(s));
        CK(cudaDeviceSynchronize());
        drop_graph(R);
        if (R.hstage) CK(cudaFreeHost(R.hstage));
        if (R.dstage) CK(cudaFree(R.dstage));
        if (R.hoff) CK(cudaFreeHost(R.hoff));
        if (R.doff) CK(cudaFree(R.doff));
        if (R.tables) CK(cudaFree(R.tables));
        R.hstage = R.dstage = R.tables = nullptr;
        R.hoff = R.doff = nullptr;
        R.cap = 0;
        const size_t sb = batch_stage_bytes(cap);
        CK(cudaMallocHost((void **)&R.hstage, sb));
        CK(cudaMalloc((void **)&R.dstage, sb));
        CK(cudaMallocHost((void **)&R.hoff, ((size_t)cap + 1) * sizeof(uint64_t)));
        CK(cudaMalloc((void **)&R.doff, ((size_t)cap + 1) * sizeof(uint64_t)));
        CK(cudaMalloc((void **)&R.tables, (size_t)cap * group::kTableBytes));
        if (!R.rt)
            CK(cudaMalloc((void **)&R.rt, (size_t)group::kRangesPerBlock * stream::kMaxBlocks *
                                              sizeof(unsigned long long)));
        R.cap = cap;
    }
    if (ncomb > R.comb_cap) {
        const uint32_t cc = std::max<uint32_t>({ncomb, R.comb_cap * 2u, 4u});
        CK(cudaStreamSynchronize(s));
        drop_graph(R);
        if (R.comb) CK(cudaFree(R.comb));
        R.comb = nullptr;
        R.comb_cap = 0;
        CK(cudaMalloc((void **)&R.comb, (size_t)cc * sizeof(group::GroupTables)));
        R.comb_cap = cc;
    }
    return EPSM_OK;
}

// Per-segment counts and list offsets for nseg pattern segments, and a hit
// list pool of pool_need entries (grown, never shrunk).
epsm_status ensure_batch_scratch(epsm_ctx *c, uint64_t nseg, uint64_t pool_need, cudaStream_t s) {
    BatchRes &R = c->batch;
    if (nseg > R.seg_cap) {
        const uint64_t cap = std::max<uint64_t>(nseg, R.seg_cap * 2);
        CK(cudaStreamSynchronize(s));
        if (R.seg_count) CK(cudaFree(R.seg_count));
        if (R.seg_off) CK(cudaFree(R.seg_off));
        R.seg_count = R.seg_off = nullptr;
        R.seg_cap = 0;
        CK(cudaMalloc((void **)&R.seg_count, cap * sizeof(uint32_t)));
        CK(cudaMalloc((void **)&R.seg_off, cap * sizeof(uint32_t)));
        R.seg_cap = cap;
        ++R.gen;
    }
    if (!R.pool_ctr) {
        CK(cudaMalloc((void **)&R.pool_ctr, sizeof(uint32_t)));
        ++R.gen;
    }
    if (pool_need > R.pool_alloc) {
        const uint64_t cap = std::max<uint64_t>(pool_need, R.pool_alloc + R.pool_alloc / 2);
        CK(cudaStreamSynchronize(s));
        if (R.pool) CK(cudaFree(R.pool));
        R.pool = nullptr;
        R.pool_alloc = 0;
        CK(cudaMalloc((void **)&R.pool, cap * sizeof(uint16_t)));
        R.pool_alloc = cap;
        ++R.gen;
    }
    return EPSM_OK;
}

group::Params batch_params(epsm_ctx *c) {
    BatchRes &R = c->batch;
    group::Params p;
    memset(&p, 0, sizeof(p));
    p.hdr = reinterpret_cast<const group::Header *>(R.dstage);
    p.jobs = reinterpret_cast<const group::JobDesc *>(R.dstage + batch_jobs_off());
    p.comb = reinterpret_cast<group::GroupTables *>(R.comb);
    p.tables = R.tables;
    p.offsets = R.doff;
    p.seg_count = R.seg_count;
    p.seg_off = R.seg_off;
    p.pool = R.pool;
    p.pool_ctr = R.pool_ctr;
    p.range_total = R.rt;
    p.err = &c->misc->err;
    p.misc = c->misc;
    return p;
}

constexpr int kTableGrid = 256;

// The four steps of a batched submission, enqueued on s.
cudaError_t enqueue_batch(epsm_ctx *c, const group::Params &p, size_t up, size_t down,
                          cudaStream_t s) {
    BatchRes &R = c->batch;
    cudaError_t e = cudaMemcpyAsync(R.dstage, R.hstage, up, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    group::build_group_tables_kernel<<<kTableGrid, 256, 0, s>>>(p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    group_kernel<<<R.grid, stream::kThreadsStream, sizeof(group::Smem), s>>>(p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    group_emit_kernel<<<R.egrid, stream::kEmitThreads, 0, s>>>(p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaMemcpyAsync(R.hoff, R.doff, down, cudaMemcpyDeviceToHost, s);
}

// Builds the submission as an explicit graph sized for the full capacity
// (upload -> table build -> filter kernel -> emission kernel -> offsets
// download);
// the two copies' sizes are set per launch.  Any failure leaves direct
// launches in use (the reason is kept in the context's error string).
void build_batch_graph(epsm_ctx *c) {
    BatchRes &R = c->batch;
    drop_graph(R);
    const group::Params p = batch_params(c);  // node arguments are copied when added
    const size_t up = batch_stage_bytes(R.cap);
    const size_t down = ((size_t)R.cap + 1) * sizeof(uint64_t);
    cudaGraph_t g = nullptr;
    cudaGraphNode_t n_up = nullptr, n_tab = nullptr, n_scan = nullptr, n_down = nullptr;
    const char *what = "cudaGraphCreate";
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e == cudaSuccess) {
        what = "memcpy node (upload)";
        e = cudaGraphAddMemcpyNode1D(&n_up, g, nullptr, 0, R.dstage, R.hstage, up,
                                     cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {
        what = "kernel node (tables)";
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof(kp));
        void *args[] = {(void *)&p};
        kp.func = (void *)group::build_group_tables_kernel;
        kp.gridDim = dim3(kTableGrid);
        kp.blockDim = dim3(256);
        kp.kernelParams = args;
        e = cudaGraphAddKernelNode(&n_tab, g, &n_up, 1, &kp);
    }
    cudaGraphNode_t n_emit = nullptr;
    if (e == cudaSuccess) {
        what = "kernel node (filter)";
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof(kp));
        void *args[] = {(void *)&p};
        kp.func = (void *)group_kernel;
        kp.gridDim = dim3(R.grid);
        kp.blockDim = dim3(stream::kThreadsStream);
        kp.sharedMemBytes = sizeof(group::Smem);
        kp.kernelParams = args;
        e = cudaGraphAddKernelNode(&n_scan, g, &n_tab, 1, &kp);
    }
    if (e == cudaSuccess) {
        what = "kernel node (emission)";
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof(kp));
        void *args[] = {(void *)&p};
        kp.func = (void *)group_emit_kernel;
        kp.gridDim = dim3(R.egrid);
        kp.blockDim = dim3(stream::kEmitThreads);
        kp.kernelParams = args;
        e = cudaGraphAddKernelNode(&n_emit, g, &n_scan, 1, &kp);
    }
    if (e == cudaSuccess) {
        what = "memcpy node (download)";
        e = cudaGraphAddMemcpyNode1D(&n_down, g, &n_emit, 1, R.hoff, R.doff, down,
                                     cudaMemcpyDeviceToHost);
    }
    if (e == cudaSuccess) {
        what = "cudaGraphInstantiate";
        e = cudaGraphInstantiate(&R.exec, g, 0);
    }
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        snprintf(c->errbuf, sizeof(c->errbuf), "batch graph: %s: %s", what, cudaGetErrorString(e));
        cudaGetLastError();
        R.exec = nullptr;
        R.graph_failed = true;
        return;
    }
    R.graph = g;
    R.up = n_up;
    R.down = n_down;
    R.graph_gen = R.gen;
}

// Window stride K of a pattern in the shared filter of its text's group (0:
// searched alone with its own variant): the largest power of two with
// K + W - 1 <= m, W = 4 for m <= 10 (K at most 4) and 8 for m >= 11 (K at
// most 8).
uint32_t shared_stride(uint32_t m) {
    if (m <= 4) return 0;
    if (m <= 6) return 2;
    if (m <= 14) return 4;
    return 8;
}

// Pairs on the same text (same pointer and length) are searched in shared
// passes: per text one group of the short patterns, run one by one on the
// staged bytes, and one group per window width of the patterns of stride
// K > 0, searched through a shared filter (more groups where a kind exceeds
// the per-group limits).
epsm_status batch_submit(epsm_ctx *c, uint32_t npairs, const uint8_t *const *texts,
                         const uint64_t *ns, const uint8_t *const *patterns, const uint32_t *ms,
                         uint64_t *positions, uint64_t capacity, cudaStream_t s) {
    using namespace group;
    // texts shared by several pairs: pairs sorted by (start, length, index),
    // so each text's pairs are one run in pair order
    std::vector<uint32_t> order(npairs);
    for (uint32_t j = 0; j < npairs; ++j) order[j] = j;
    std::sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
        if (texts[a] != texts[b]) return (uintptr_t)texts[a] < (uintptr_t)texts[b];
        if (ns[a] != ns[b]) return ns[a] < ns[b];
        return a < b;
    });
    std::vector<uint32_t> runs;  // run starts in `order`, plus npairs
    runs.reserve(npairs + 1);
    for (uint32_t k = 0; k < npairs; ++k)
        if (k == 0 || texts[order[k]] != texts[order[k - 1]] || ns[order[k]] != ns[order[k - 1]])
            runs.push_back(k);
    runs.push_back(npairs);
    std::vector<uint32_t> kstr(npairs, 0u);
    std::vector<uint8_t> multi(npairs, 0);
    for (size_t r = 0; r + 1 < runs.size(); ++r) {
        if (runs[r + 1] - runs[r] < 2) continue;
        for (uint32_t k = runs[r]; k < runs[r + 1]; ++k) {
            const uint32_t j = order[k];
            kstr[j] = shared_stride(ms[j]);
            multi[j] = 1;
        }
    }
    // jobs (pairs with at least one stage), in pair order; shared patterns use
    // the numbering with start offset 0 of the window variants
    std::vector<int32_t> jidx(npairs, -1);
    std::vector<JobDesc> kept;
    kept.reserve(npairs);
    uint64_t jst = 0;
    uint64_t starts = 0;  // valid starts over all pairs: a bound on the hits
    uint32_t ntab = 0;
    for (uint32_t i = 0; i < npairs; ++i) {
        const uint32_t m = ms[i];
        JobDesc D;
        memset(&D, 0, sizeof(D));
        D.job = make_job(texts[i], ns[i], pack_pattern(patterns[i], m));
        D.job.pat.kbits = c->tune[text_bucket(ns[i])][m].kbits;
        // shared patterns are numbered like the window variants (offset 0);
        // short patterns of a shared text run the direct compare
        // (the strided block variant is single-search only: its batch form is
        // the plain block variant)
        const Tune &T = c->tune[text_bucket(ns[i])][m];
        const int vt = T.variant == V_BLOCK8S ? V_BLOCK8 : T.variant;
        D.variant = (uint32_t)(kstr[i] ? V_PREFIX4 : multi[i] ? V_DIRECT : vt);
        const uint64_t nst = stages_for(D.job.delta, ns[i], m, (int)D.variant);
        if (nst == 0) continue;
        D.pair = i;
        D.stage0 = jst;
        D.nstages = nst;
        D.off = variant_offset((int)D.variant);
        D.kstride = kstr[i];
        D.table = (!kstr[i] && D.variant == (uint32_t)V_BLOCK8) ? ntab++ : kNone;
        jidx[i] = (int32_t)kept.size();
        kept.push_back(D);
        jst += nst;
        starts += ns[i] - m + 1u;
    }
    const uint32_t nj = (uint32_t)kept.size();
    BatchRes &RB = c->batch;
    RB.pend_jidx = jidx;
    RB.pend_npairs = npairs;
    RB.pend_nj = nj;
    RB.pend_capacity = capacity;
    if (nj == 0) return mark_done(c, s);
    // groups: per text and kind, shared patterns up to kMaxShared / kMaxEnt
    // entries or individual ones up to kIndivMax per group
    std::vector<GroupDesc> groups;
    std::vector<uint32_t> gjobs;
    gjobs.reserve(nj);
    uint32_t ncomb = 0;
    uint64_t gst = 0;
    // Each text's patterns form up to three kinds of group, searched as
    // separate passes over the text: the short ones (direct compare), the
    // shared filter with 4-byte windows and the one with 8-byte windows.  Kept
    // apart, each pass runs at the pace of its own kind instead of the slowest
    // kind's (the short patterns' many hits hold up a combined pass).
    std::vector<uint32_t> cls[3];
    for (size_t r = 0; r + 1 < runs.size(); ++r) {
        for (auto &v : cls) v.clear();
        for (uint32_t k = runs[r]; k < runs[r + 1]; ++k) {
            const uint32_t pi = order[k];
            if (jidx[pi] < 0) continue;
            cls[!kstr[pi] ? 0 : ms[pi] < kW8Min ? 1 : 2].push_back((uint32_t)jidx[pi]);
        }
        for (int kc = 0; kc < 3; ++kc) {
            const std::vector<uint32_t> &L = cls[kc];
            size_t pos = 0;
            while (pos < L.size()) {
                GroupDesc G;
                memset(&G, 0, sizeof(G));
                G.job0 = (uint32_t)gjobs.size();
                uint64_t nst = 0;
                uint32_t kmin = 0;
                if (kc == 0) {
                    while (pos < L.size() && G.nindiv < (uint32_t)kIndivMax) {
                        const uint32_t jj = L[pos++];
                        ++G.nindiv;
                        gjobs.push_back(jj);
                        nst = std::max(nst, kept[jj].nstages);
                    }
                } else {
                    while (pos < L.size() && G.nshared < (uint32_t)kMaxShared &&
                           G.nent + kept[L[pos]].kstride <= (uint32_t)kMaxEnt) {
                        JobDesc &D = kept[L[pos++]];
                        D.ent0 = G.nent;
                        G.nent += D.kstride;
                        ++G.nshared;
                        gjobs.push_back((uint32_t)(&D - kept.data()));
                        nst = std::max(nst, D.nstages);
                        kmin = kmin ? std::min(kmin, D.kstride) : D.kstride;
                    }
                }
                const JobDesc &D0 = kept[gjobs[G.job0]];
                G.text = D0.job;
                G.chunk_full0 = (D0.job.delta + 15u) / 16u;
                G.chunk_full1 = D0.job.lim / 16u;
                G.gstage0 = gst;
                G.nstages = nst;
                G.cfg = kc == 2 ? kmin : (kmin << 8);
                G.comb = (G.nshared || G.nindiv > 1u) ? ncomb++ : kNone;
                gst += nst;
                groups.push_back(G);
            }
        }
    }
    const uint32_t ng = (uint32_t)groups.size();
    epsm_status st;
    if ((st = ensure_batch(c, std::max(nj, ng), ncomb, s)) != EPSM_OK) return st;
    BatchRes &R = c->batch;
    if (R.grid == 0) R.grid = batch_grid(c->sms);
    if (R.egrid == 0) R.egrid = emit_grid(c->sms);
    if (R.grid == 0 || R.egrid == 0) return EPSM_ERR_CUDA;
    Header &H = *reinterpret_cast<Header *>(R.hstage);
    memset(&H, 0, sizeof(H));
    H.ngroups = ng;
    H.njobs = nj;
    H.gstages = gst;
    H.jstages = jst;
    // emit ranges, claimed dynamically by the emission kernel's blocks: many
    // (dense ranges take longer than sparse ones), each at least one batch of
    // 256 stages (one per emission thread), at most the range-total buffer
    const uint64_t per_batch = (uint64_t)stream::kEmitThreads;
    const uint64_t nr_want = std::max<uint64_t>(
        1, std::min<uint64_t>(jst / per_batch, (uint64_t)kRangesPerBlock * stream::kMaxBlocks));
    H.range_stages = (jst + nr_want - 1) / nr_want;
    H.nranges = (uint32_t)((jst + H.range_stages - 1) / H.range_stages);
    H.capacity = capacity;
    H.positions = positions;
    H.emit = capacity > 0 ? 1u : 0u;
    const size_t goff = batch_jobs_off() + align16((size_t)nj * sizeof(JobDesc));
    const size_t gjoff = goff + align16((size_t)ng * sizeof(GroupDesc));
    H.groups = reinterpret_cast<const GroupDesc *>(R.dstage + goff);
    H.group_jobs = reinterpret_cast<const uint32_t *>(R.dstage + gjoff);
    memcpy(R.hstage + batch_jobs_off(), kept.data(), nj * sizeof(JobDesc));
    memcpy(R.hstage + goff, groups.data(), ng * sizeof(GroupDesc));
    memcpy(R.hstage + gjoff, gjobs.data(), gjobs.size() * sizeof(uint32_t));
    // hit lists: at most min(capacity, starts) entries, plus the unused tail of
    // each warp's last pool chunk
    H.pool_cap = capacity > 0 ? std::min<uint64_t>(capacity, starts) +
                                    (uint64_t)R.grid * stream::kConsumerWarps * kPoolChunk
                              : 0;
    if ((st = ensure_batch_scratch(c, jst * stream::kConsumerWarps, H.pool_cap, s)) != EPSM_OK) return st;
    if ((st = order_after_previous(c, s)) != EPSM_OK) return st;
    const size_t up = gjoff + gjobs.size() * sizeof(uint32_t);
    const size_t down = ((size_t)nj + 1) * sizeof(uint64_t);
    if (!R.graph_failed && (!R.exec || R.graph_gen != R.gen)) build_batch_graph(c);
    bool launched = false;
    if (!R.graph_failed && R.exec) {
        if (cudaGraphExecMemcpyNodeSetParams1D(R.exec, R.up, R.dstage, R.hstage, up,
                                               cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaGraphExecMemcpyNodeSetParams1D(R.exec, R.down, R.hoff, R.doff, down,
                                               cudaMemcpyDeviceToHost) == cudaSuccess &&
            cudaGraphLaunch(R.exec, s) == cudaSuccess) {
            launched = true;
        } else {
            cudaGetLastError();
            R.graph_failed = true;
        }
    }
    if (!launched) CK(enqueue_batch(c, batch_params(c), up, down, s));
    c->launches += 3;  // table build + batched filter + emission
    CK(cudaMemcpyAsync(c->hmisc, c->misc, sizeof(DevMisc), cudaMemcpyDeviceToHost, s));
    return mark_done(c, s);
}

// Results of the batch submitted last on c, once its work has completed
// (the context's event): pair offsets and the status.
epsm_status batch_complete(epsm_ctx *c, uint64_t *offsets) {
    BatchRes &R = c->batch;
    const uint32_t npairs = R.pend_npairs;
    if (R.pend_nj == 0) {
        for (uint32_t i = 0; i <= npairs; ++i) offsets[i] = 0;
        return EPSM_OK;
    }
    const uint32_t err = c->hmisc->err;
    if (err) {
        CK(cudaMemsetAsync(&c->misc->err, 0, sizeof(uint32_t), c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    // job offsets -> pair offsets; pairs without stages own an empty range at
    // the next pair's offset
    const std::vector<int32_t> &jidx = R.pend_jidx;
    offsets[npairs] = R.hoff[R.pend_nj];
    for (uint32_t i = npairs; i-- > 0;)
        offsets[i] = jidx[i] >= 0 ? R.hoff[jidx[i]] : offsets[i + 1];
    if (err & kErrTimeout) return EPSM_ERR_TIMEOUT;
    return offsets[npairs] > R.pend_capacity ? EPSM_ERR_CAPACITY : EPSM_OK;
}

epsm_status batch_impl(epsm_ctx *c, uint32_t npairs, const uint8_t *const *texts,
                       const uint64_t *ns, const uint8_t *const *patterns, const uint32_t *ms,
                       uint64_t *positions, uint64_t capacity, uint64_t *offsets,
                       cudaStream_t s) {
    epsm_status st = batch_submit(c, npairs, texts, ns, patterns, ms, positions, capacity, s);
    if (st != EPSM_OK) return st;
    CK(cudaEventSynchronize(c->ev));
    return batch_complete(c, offsets);
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

EPSM_API epsm_status epsm_create(epsm_ctx **out, int device, uint64_t flags) {
    (void)flags;
    if (!out) return EPSM_ERR_ARG;
    *out = nullptr;
    epsm_ctx *c = new (std::nothrow) epsm_ctx();
    if (!c) return EPSM_ERR_NOMEM;
    c->errbuf[0] = 0;
    c->device = device;
    for (int b = 0; b < EPSM_TEXT_BUCKETS; ++b)
        for (uint32_t m = 0; m <= EPSM_MAX_M; ++m)
            c->tune[b][m] = Tune{m ? default_variant(m) : 0, stream::kDefaultShape, (uint32_t)kHashBitsDefault};
    auto fail = [&](epsm_status st) {
        epsm_destroy(c);
        return st;
    };
    cudaError_t e;
    if ((e = cudaSetDevice(device)) != cudaSuccess) return fail(cuda_fail(nullptr, e, "cudaSetDevice"));
    if ((e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess)
        return fail(cuda_fail(nullptr, e, "attr"));
    if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess)
        return fail(cuda_fail(nullptr, e, "stream"));
    if ((e = cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming)) != cudaSuccess)
        return fail(cuda_fail(nullptr, e, "event"));
    if ((e = cudaMalloc(&c->misc, sizeof(DevMisc))) != cudaSuccess) return fail(cuda_fail(nullptr, e, "misc"));
    if ((e = cudaMallocHost(&c->hmisc, sizeof(DevMisc))) != cudaSuccess)
        return fail(cuda_fail(nullptr, e, "hmisc"));
    if ((e = cudaMemset(c->misc, 0, sizeof(DevMisc))) != cudaSuccess) return fail(cuda_fail(nullptr, e, "memset"));
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(cuda_fail(nullptr, e, "sync"));
    *out = c;
    return EPSM_OK;
}

EPSM_API epsm_status epsm_destroy(epsm_ctx *c) {
    if (!c) return EPSM_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaDeviceSynchronize();
    if (c->misc) cudaFree(c->misc);
    if (c->hmisc) cudaFreeHost(c->hmisc);
    free_batch(c->batch);
    if (c->seg_count) cudaFree(c->seg_count);
    if (c->range_total) cudaFree(c->range_total);
    if (c->seg_mask) cudaFree(c->seg_mask);
    if (c->dtext) cudaFree(c->dtext);
    if (c->dpos) cudaFree(c->dpos);
    if (c->tail) cudaFree(c->tail);
    if (c->copy_ev) cudaEventDestroy(c->copy_ev);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->ev) cudaEventDestroy(c->ev);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return EPSM_OK;
}

EPSM_API const char *epsm_status_str(epsm_status s) {
    switch (s) {
        case EPSM_OK: return "EPSM_OK";
        case EPSM_ERR_ARG: return "EPSM_ERR_ARG";
        case EPSM_ERR_CAPACITY: return "EPSM_ERR_CAPACITY";
        case EPSM_ERR_CUDA: return "EPSM_ERR_CUDA";
        case EPSM_ERR_NOMEM: return "EPSM_ERR_NOMEM";
        case EPSM_ERR_TIMEOUT: return "EPSM_ERR_TIMEOUT";
        default: return "EPSM_ERR_UNKNOWN";
    }
}

EPSM_API const char *epsm_last_error(epsm_ctx *c) { return c ? c->errbuf : ""; }

EPSM_API epsm_status epsm_search_async(epsm_ctx *c, const uint8_t *text, uint64_t n,
                                       const uint8_t *pattern, uint32_t m, uint64_t *positions,
                                       uint64_t capacity, uint64_t *count_dev, void *stream) {
    if (!c) return EPSM_ERR_ARG;
    DeviceGuard dg(c->device);
    if (!dg.ok) return EPSM_ERR_CUDA;
    return search_async_impl(c, EPSM_VARIANT_AUTO, text, n, pattern, m, positions, capacity,
                             count_dev, stream, nullptr);
}

EPSM_API epsm_status epsm_search_variant(epsm_ctx *c, int variant, const uint8_t *text,
                                         uint64_t n, const uint8_t *pattern, uint32_t m,
                                         uint64_t *positions, uint64_t capacity,
                                         uint64_t *count_dev, void *stream) {
    if (!c) return EPSM_ERR_ARG;
    DeviceGuard dg(c->device);
    if (!dg.ok) return EPSM_ERR_CUDA;
    return search_async_impl(c, variant, text, n, pattern, m, positions, capacity, count_dev,
                             stream, nullptr);
}

EPSM_API epsm_status epsm_search(epsm_ctx *c, const uint8_t *text, uint64_t n,
                                 const uint8_t *pattern, uint32_t m, uint64_t *positions,
                                 uint64_t capacity, uint64_t *count, void *stream) {
    if (!c || !count) return EPSM_ERR_ARG;
    DeviceGuard dg(c->device);
    if (!dg.ok) return EPSM_ERR_CUDA;
    epsm_status st = search_async_impl(c, EPSM_VARIANT_AUTO, text, n, pattern, m, positions,
                                       capacity, &c->misc->count, stream, nullptr);
    if (st != EPSM_OK) return st;
    uint32_t err = 0;
    if ((st = read_misc(c, pick_stream(c, stream), &err)) != EPSM_OK) return st;
    *count = c->hmisc->count;
    if (err & kErrTimeout) return EPSM_ERR_TIMEOUT;
    return *count > capacity ? EPSM_ERR_CAPACITY : EPSM_OK;
}

// Diagnostic: one warp waits, bounded by limit_ns, for a device flag that
// nothing sets, as every wait of the search kernels is bounded; when the
// limit passes it sets the context's timeout bit, which the next epsm_sync
// reports.  Shows that a wait that gives up leaves the context usable.
__global__ void wait_probe_kernel(const uint32_t *flag, uint32_t *err, uint64_t limit_ns) {
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        uint32_t v;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v) return;
        if (globaltimer_ns() - t0 > limit_ns) {
            if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
            return;
        }
        __nanosleep(1000);
    }
}

EPSM_API epsm_status epsm_wait_probe(epsm_ctx *c, uint64_t limit_ns, void *stream) {
    if (!c || limit_ns == 0 || limit_ns > 1000000000ull) return EPSM_ERR_ARG;
    DeviceGuard dg(c->device);
    if (!dg.ok) return EPSM_ERR_CUDA;
    cudaStream_t s = pick_stream(c, stream);
    epsm_status st = order_after_previous(c, s);
    if (st != EPSM_OK) return st;
    // the flag: a scratch word nothing sets
    CK(cudaMemsetAsync(&c->misc->probe, 0, sizeof(uint32_t), s));
    wait_probe_kernel<<<1, 32, 0, s>>>(&c->misc->probe, &c->misc->err, limit_ns);
    CK(cudaGetLastError());
    c->launches += 1;
    return mark_done(c, s);
}

EPSM_API epsm_status epsm_sync(epsm_ctx *c, void *stream) {
    if (!c) return EPSM_ERR_ARG;
    DeviceGuard dg(c->device);
    if (!dg.ok) return EPSM_ERR_CUDA;
    uint32_t err = 0;
    epsm_status st = read_misc(c, pick_stream(c, stream), &err);
    if (st != EPSM_OK) return st;
    if (err & kErrTimeout) return EPSM_ERR_TIMEOUT;
    if (err & kErrCapacity) return EPSM_ERR_CAPACITY;
    return EPSM_OK;
}

EPSM_API epsm_status epsm_search_batch(epsm_ctx *c, uint32_t npairs, const uint8_t *const *texts,
                                       const uint64_t *ns, const uint8_t *const *patterns,
                                       const uint32_t *ms, uint64_t *positions, uint64_t capacity,
                                       uint64_t *offsets, void *stream) {
    if (!c || !offsets) return EPSM_ERR_ARG;
    if (npairs == 0) {
        offsets[0] = 0;
        return EPSM_OK;
    }
    if (!texts || !ns || !patterns || !ms) return EPSM_ERR_ARG;
    if (capacity > 0 && !positions) return EPSM_ERR_ARG;
    DeviceGuard dg(c->device);
    if (!dg.ok) return EPSM_ERR_CUDA;
    for (uint32_t i = 0; i < npairs; ++i) {
        if (ms[i] == 0 || ms[i] > EPSM_MAX_M || !patterns[i]) return EPSM_ERR_ARG;
        if (ns[i] > 0 && !texts[i]) return EPSM_ERR_ARG;
    }
    return batch_impl(c, npairs, texts, ns, patterns, ms, positions, capacity, offsets,
                      pick_stream(c, stream));
}

EPSM_API epsm_status epsm_search_host(epsm_ctx *c, const uint8_t *text_host, uint64_t n,
                                      const uint8_t *patterns_host, const uint32_t *ms,
                                      uint32_t npat, uint64_t *positions_host, uint64_t capacity,
                                      uint64_t *offsets_host) {
    if (!c || !offsets_host || (n > 0 && !text_host)) return EPSM_ERR_ARG;
    if (npat > 0 && (!patterns_host || !ms)) return EPSM_ERR_ARG;
    if (capacity > 0 && !positions_host) return EPSM_ERR_ARG;
    for (uint32_t k = 0; k < npat; ++k)
        if (ms[k] == 0 || ms[k] > EPSM_MAX_M_LONG) return EPSM_ERR_ARG;
    DeviceGuard dg(c->device);
    if (!dg.ok) return EPSM_ERR_CUDA;
    cudaStream_t s = c->stream;
    if (n + 16 > c->dtext_cap) {
        CK(cudaStreamSynchronize(s));
        if (c->dtext) CK(cudaFree(c->dtext));
        c->dtext = nullptr;
        c->dtext_cap = 0;
        CK(cudaMalloc(&c->dtext, n + 16));
        c->dtext_cap = n + 16;
    }
    if (capacity > c->dpos_cap) {
        CK(cudaStreamSynchronize(s));
        if (c->dpos) CK(cudaFree(c->dpos));
        c->dpos = nullptr;
        c->dpos_cap = 0;
        CK(cudaMalloc(&c->dpos, capacity * sizeof(uint64_t)));
        c->dpos_cap = capacity;
    }
    epsm_status st = order_after_previous(c, s);
    if (st != EPSM_OK) return st;
    if (n) CK(cudaMemcpyAsync(c->dtext, text_host, n, cudaMemcpyHostToDevice, s));
    if (!c->copy_stream) {
        CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->copy_ev, cudaEventDisableTiming));
    }
    // one single search per pattern (the kernels of epsm_search), each writing
    // its positions right after the previous pattern's; the count comes back
    // after each search, and that pattern's positions are copied back on a
    // second stream while the next pattern is searched
    uint64_t off = 0;
    uint64_t p0 = 0;
    for (uint32_t k = 0; k < npat; ++k) {
        offsets_host[k] = off;
        const uint64_t room = off < capacity ? capacity - off : 0;
        st = search_async_impl(c, EPSM_VARIANT_AUTO, c->dtext, n, patterns_host + p0, ms[k],
                               room ? c->dpos + off : nullptr, room, &c->misc->count, s, nullptr);
        if (st != EPSM_OK) return st;
        uint32_t err = 0;
        if ((st = read_misc(c, s, &err)) != EPSM_OK) return st;
        if (err & kErrTimeout) return EPSM_ERR_TIMEOUT;
        const uint64_t cnt = c->hmisc->count;
        const uint64_t got = std::min<uint64_t>(cnt, room);
        if (got) {
            CK(cudaEventRecord(c->copy_ev, s));
            CK(cudaStreamWaitEvent(c->copy_stream, c->copy_ev, 0));
            CK(cudaMemcpyAsync(positions_host + off, c->dpos + off, got * sizeof(uint64_t),
                               cudaMemcpyDeviceToHost, c->copy_stream));
        }
        off += cnt;
        p0 += ms[k];
    }
    offsets_host[npat] = off;
    CK(cudaStreamSynchronize(c->copy_stream));
    return off > capacity ? EPSM_ERR_CAPACITY : EPSM_OK;
}

EPSM_API int epsm_variant_for(epsm_ctx *c, uint32_t m) {
    if (!c || m == 0 || m > EPSM_MAX_M) return 0;
    return c->tune[EPSM_TEXT_BUCKETS - 1][m].variant;
}

EPSM_API epsm_status epsm_set_variant(epsm_ctx *c, uint32_t m, int variant) {
    if (!c || m == 0 || m > EPSM_MAX_M) return EPSM_ERR_ARG;
    if (!variant_covers(variant, m)) return EPSM_ERR_ARG;
    for (int b = 0; b < EPSM_TEXT_BUCKETS; ++b) c->tune[b][m].variant = variant;
    return EPSM_OK;
}

EPSM_API epsm_status epsm_set_tuning(epsm_ctx *c, int bucket, uint32_t m, int variant, int shape,
                                     uint32_t kbits) {
    if (!c || m == 0 || m > EPSM_MAX_M || bucket < -1 || bucket >= EPSM_TEXT_BUCKETS) return EPSM_ERR_ARG;
    if (variant != EPSM_VARIANT_AUTO && !variant_covers(variant, m)) return EPSM_ERR_ARG;
    if (shape < -1 || shape >= stream::kShapes) return EPSM_ERR_ARG;
    if (kbits != 0 && (kbits < EPSM_KBITS_MIN || kbits > EPSM_KBITS_MAX)) return EPSM_ERR_ARG;
    for (int b = 0; b < EPSM_TEXT_BUCKETS; ++b) {
        if (bucket >= 0 && b != bucket) continue;
        Tune &T = c->tune[b][m];
        if (variant != EPSM_VARIANT_AUTO) T.variant = variant;
        if (shape >= 0) T.shape = shape;
        if (kbits) T.kbits = kbits;
    }
    return EPSM_OK;
}

EPSM_API epsm_status epsm_get_tuning(epsm_ctx *c, int bucket, uint32_t m, int *variant, int *shape,
                                     uint32_t *kbits) {
    if (!c || m == 0 || m > EPSM_MAX_M || bucket < 0 || bucket >= EPSM_TEXT_BUCKETS) return EPSM_ERR_ARG;
    const Tune &T = c->tune[bucket][m];
    if (variant) *variant = T.variant;
    if (shape) *shape = T.shape;
    if (kbits) *kbits = T.kbits;
    return EPSM_OK;
}

EPSM_API uint64_t epsm_launch_count(epsm_ctx *c) { return c ? c->launches : 0; }

EPSM_API int epsm_batch_uses_graph(epsm_ctx *c) {
    return c && c->batch.exec != nullptr && !c->batch.graph_failed ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Search without any allocation (epsm_search_static).
//
// For callers that cannot allocate device memory at all: code running where
// cudaMalloc is forbidden or unavailable (inside a framework that owns every
// allocation through its own pool, a real-time loop where an allocation could
// stall or fail, or a plug-in whose host application pre-sizes all memory).
// The streaming kernel's scratch (segment counts and masks, block status
// words) lives in the fixed array below instead of in a context.  The array
// is reserved on every GPU that loads this library until the process exits.
// ---------------------------------------------------------------------------

namespace {

// stages_for: (delta + n - m - off) / stage + 1 with delta <= 15 and off >= -15
constexpr uint64_t kStaticMaxStages =
    (EPSM_STATIC_MAX_TEXT + 15u + 15u) / stream::kStageBytes + 1u;
constexpr uint64_t kStaticMaxSegs = kStaticMaxStages * stream::kConsumerWarps;
constexpr uint64_t kStaticCountBytes = kStaticMaxSegs * sizeof(uint32_t);
constexpr uint64_t kStaticMaskBytes = kStaticMaxSegs * stream::kSegChunks * sizeof(uint16_t);
constexpr uint64_t kStaticMiscBytes = 256 + kMaxRanges * 8;  // DevMisc + range totals
constexpr uint64_t kStaticBytes = kStaticMiscBytes + kStaticCountBytes + kStaticMaskBytes;

// In host code `g_static_scratch` only names the symbol; its device address
// comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) uint8_t g_static_scratch[kStaticBytes];

struct StaticDevice {
    bool ready = false;
    uint8_t *base = nullptr;  // device address of g_static_scratch on this device, past misc
    DevMisc *misc = nullptr;
    int sms = 0;
};

constexpr int kMaxStaticDevices = 64;
std::mutex g_static_mu;
StaticDevice g_static_dev[kMaxStaticDevices];

}  // namespace

EPSM_API epsm_status epsm_search_static(const uint8_t *text, uint64_t n, const uint8_t *pattern,
                                        uint32_t m, uint64_t *positions, uint64_t capacity,
                                        uint64_t *result_dev, void *stream) {
    if (!pattern || !result_dev || m == 0 || m > EPSM_MAX_M) return EPSM_ERR_ARG;
    if (n > 0 && !text) return EPSM_ERR_ARG;
    if (capacity > 0 && !positions) return EPSM_ERR_ARG;
    if (n > EPSM_STATIC_MAX_TEXT) return EPSM_ERR_ARG;  // beyond the fixed scratch
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxStaticDevices)
        return EPSM_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_static_mu);
    StaticDevice &D = g_static_dev[dev];
    if (!D.ready) {
        // one-time set-up on this device (the device is current)
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) return EPSM_ERR_CUDA;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return EPSM_ERR_CUDA;
        // the claim tickets, done counters and range totals must start at
        // zero; the clearing completes before the device is marked ready, so
        // a first call on one stream cannot race a later call on another
        if (cudaMemsetAsync(ptr, 0, kStaticMiscBytes, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return EPSM_ERR_CUDA;
        D.base = static_cast<uint8_t *>(ptr) + kStaticMiscBytes;
        D.misc = static_cast<DevMisc *>(ptr);
        D.sms = sms;
        D.ready = true;
    }
    const int v = default_variant(m);
    stream::StreamParams p;
    memset(&p, 0, sizeof(p));
    p.job = make_job(text, n, pack_pattern(pattern, m));
    p.nstages = stages_for(p.job.delta, n, m, v);
    if (p.nstages > kStaticMaxStages) return EPSM_ERR_ARG;  // (cannot happen for n <= the maximum)
    // result_dev[0] = count, result_dev[1] = device error bits; the error word
    // must start at zero
    if (cudaMemsetAsync(result_dev, 0, 2 * sizeof(uint64_t), s) != cudaSuccess) return EPSM_ERR_CUDA;
    if (n < m) return EPSM_OK;
    p.chunk_full0 = (p.job.delta + 15u) / 16u;
    p.chunk_full1 = p.job.lim / 16u;
    p.emit = capacity > 0 ? 1 : 0;
    p.positions = positions;
    p.capacity = capacity;
    p.count_out = result_dev;
    p.seg_count = reinterpret_cast<uint32_t *>(D.base);
    p.seg_mask = reinterpret_cast<uint16_t *>(D.base + kStaticCountBytes);
    p.err = reinterpret_cast<uint32_t *>(result_dev + 1);
    p.misc = D.misc;
    p.range_total = reinterpret_cast<unsigned long long *>(reinterpret_cast<uint8_t *>(D.misc) + 256);
    if (launch_stream(D.sms, v, m, stream::kDefaultShape, p, s) != cudaSuccess) return EPSM_ERR_CUDA;
    return EPSM_OK;
}

#include "epsm_serve.inc"
