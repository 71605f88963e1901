// Device building blocks of the exact short-pattern scan (sm_103a).
//
// A search is the problem of Section 1: all s in [0, n-m] with t[s..s+m) == p.
// The text is processed in tiles; each warp streams 16-byte chunks with
// coalesced vector loads, a per-variant filter marks candidate starts (the
// Section 3 procedures re-thought for 32-bit lanes), candidates are verified,
// and the hits are compacted in order (see epsm_stream.cuh).
//
// Coordinates.  `base` is the text pointer rounded down to 16 bytes and
// `delta` = text - base.  An internal position P addresses base[P]; the user
// position is s = P - delta.  Valid starts are delta <= P <= pmax = delta+n-m.
// Chunk c covers internal bytes [16c, 16c+16).  Only bytes inside
// [delta, delta+n) are ever read: whole-chunk vector loads are used when the
// chunk lies inside, byte loads at the two ragged ends.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace epsm {

// Filter-soundness build (-DEPSM_FILTER_SOUNDNESS=1, a test build): the
// single-search filters pass every start, so that the verification alone
// decides; its results must equal those of the normal build.
#ifndef EPSM_FILTER_SOUNDNESS
#define EPSM_FILTER_SOUNDNESS 0
#endif
constexpr bool kSoundness = EPSM_FILTER_SOUNDNESS != 0;

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kFull = 0xffffffffu;

// Variants (see include/epsm.h).
constexpr int V_DIRECT = 1;
constexpr int V_PREFIX4 = 2;
constexpr int V_PREFIX8 = 3;
constexpr int V_BLOCK8 = 4;
constexpr int V_BLOCK4 = 5;
constexpr int V_CODE2 = 6;
constexpr int V_ADAPT = 7;
constexpr int V_BLOCK8S = 8;

// Block fingerprint table (Section 3.4): a bit table of 2^k slots.  The paper
// takes k = 11; here k is a parameter of the search (1 <= k <= kHashBitsMax,
// default kHashBitsDefault): a wider table makes false fingerprint matches of
// the text's blocks rarer at no cost in shared memory (2^14 bits = 2 KiB).
constexpr int kHashBitsMax = 14;
constexpr int kHashBitsDefault = 14;
constexpr int kTableWords = (1 << kHashBitsMax) / 32;  // uint32 words of the bit table

// Error bits of the device error word.
constexpr uint32_t kErrTimeout = 1u;   // a look-back wait gave up
constexpr uint32_t kErrCapacity = 2u;  // an occurrence did not fit in the output

struct Pattern {
    uint32_t w[8];  // p packed little-endian, zero padded (the paper's blocks P_i, Section 2)
    uint32_t m;
    // Smallest period q of p (p[i] == p[i+q] for all i < m-q) when q <= 8 and
    // m <= 32, else 0.  If s is an occurrence, s+q is one iff the text's bytes
    // [s+m-q, s+m) equal p's last q bytes (the other m-q already match by
    // periodicity); the block variants use this to confirm the candidates of
    // a run in one 8-byte compare each.
    uint32_t q;
    uint32_t tl, th;  // p's last 8 bytes (m >= 8), little-endian
    uint32_t kbits;   // fingerprint width k of the block variants' table
};

struct SearchJob {
    const uint8_t *base;  // text rounded down to 16 bytes
    uint64_t delta;       // text - base
    uint64_t lim;         // delta + n: first internal byte past the text
    int64_t pmax;         // delta + n - m: last valid internal start
    Pattern pat;
};

// ---------------------------------------------------------------------------
// memory helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint4 ldg_v4(const uint8_t *p) {
    uint4 r;
    asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}

__device__ __forceinline__ uint32_t ldg_u32(const uint8_t *p) {
    uint32_t r;
    asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
}

__device__ __forceinline__ uint32_t ldg_u8(const uint8_t *p) {
    uint16_t r;
    asm volatile("ld.global.nc.u8 %0, [%1];" : "=h"(r) : "l"(p));
    return r;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The 16-byte chunk c of the text; bytes outside [delta, lim) read as 0.
__device__ __forceinline__ uint4 load_chunk(const SearchJob &J, uint64_t c) {
    uint64_t b0 = c * 16ull;
    if (b0 >= J.delta && b0 + 16ull <= J.lim) return ldg_v4(J.base + b0);
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if (b0 + 16ull > J.delta && b0 < J.lim) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            uint64_t b = b0 + (uint64_t)i;
            if (b >= J.delta && b < J.lim) w[i >> 2] |= ldg_u8(J.base + b) << (8 * (i & 3));
        }
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// 4-byte word widx of the text; bytes outside [delta, lim) read as 0.
__device__ __forceinline__ uint32_t load_word(const SearchJob &J, uint64_t widx) {
    uint64_t b0 = widx * 4ull;
    if (b0 >= J.delta && b0 + 4ull <= J.lim) return ldg_u32(J.base + b0);
    uint32_t w = 0u;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint64_t b = b0 + (uint64_t)i;
        if (b >= J.delta && b < J.lim) w |= ldg_u8(J.base + b) << (8 * i);
    }
    return w;
}

// Programmatic dependent launch (kernels launched with the programmatic
// stream serialization attribute may start before the previous kernel of the
// stream ends): wait until that kernel has completed and its writes are
// visible (returns at once when there is none), and let the next kernel be
// scheduled (it waits for this one in the same way before it reads anything).
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Sets an error bit; reads first so that many reporters of the same
// condition do not all queue an atomic on one word.
__device__ __forceinline__ void set_err(uint32_t *err, uint32_t bit) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(err) : "memory");
    if (!(v & bit)) atomicOr(err, bit);
}

// ---------------------------------------------------------------------------
// packed-byte helpers (the wscmp idea of Section 3.1 on 32-bit lanes)
// ---------------------------------------------------------------------------

// Exact zero-byte mask: bit 8b+7 set iff byte b of x is zero.
__device__ __forceinline__ uint32_t zero_bytes(uint32_t x) {
    uint32_t y = (x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu;
    return ~(y | x | 0x7F7F7F7Fu);
}

// Nonzero iff some byte of x is zero (exact as a test, not as a mask).
__device__ __forceinline__ uint32_t has_zero_byte(uint32_t x) {
    return (x - 0x01010101u) & ~x & 0x80808080u;
}

// Bits 7,15,23,31 of z -> bits 0..3.
__device__ __forceinline__ uint32_t nibble_of(uint32_t z) {
    return ((z >> 7) * 0x10204080u) >> 28;
}

// Byte j of w replicated four times: the broadcast word (p_j)^4 (Section 3.2, table B).
__device__ __forceinline__ uint32_t bcast_byte(uint32_t w, int j) {
    return __byte_perm(w, 0u, (uint32_t)(j * 0x1111));
}

// Multiplicative (Fibonacci) hash of an 8-byte block to k bits (1 <= k <= 14).
__device__ __forceinline__ uint32_t block_hash(uint32_t lo, uint32_t hi, uint32_t k) {
    return (lo * 0x9E3779B1u + hi * 0x85EBCA77u) >> (32u - k);
}

// Slot h of a fingerprint bit table.
__device__ __forceinline__ uint32_t table_bit(const uint32_t *table, uint32_t h) {
    return (table[h >> 5] >> (h & 31u)) & 1u;
}

// Mask of the bytes of pattern word i that belong to the pattern.
__device__ __forceinline__ uint32_t word_mask(uint32_t m, uint32_t i) {
    uint32_t rem = m - 4u * i;
    return rem >= 4u ? 0xFFFFFFFFu : ((1u << (8u * rem)) - 1u);
}

// Naive check (Section 3, "check position"): t[P..P+m) == p, read from global.
__device__ __noinline__ bool verify_global(const SearchJob &J, int64_t P) {
    uint64_t a = (uint64_t)P >> 2;
    uint32_t sh = ((uint32_t)P & 3u) * 8u;
    uint32_t m = J.pat.m;
    uint32_t nw = (m + 3u) >> 2;
    uint32_t cur = load_word(J, a);
    for (uint32_t i = 0; i < nw; ++i) {
        uint32_t nxt = (sh != 0u || i + 1u < nw) ? load_word(J, a + i + 1u) : 0u;
        uint32_t win = __funnelshift_r(cur, nxt, sh);
        if ((win ^ J.pat.w[i]) & word_mask(m, i)) return false;
        cur = nxt;
    }
    return true;
}

// Where a candidate can be checked from: the staged stage buffer holds the
// text's internal bytes [sbase, sbase + span) when `inside` is set.
struct StagedText {
    const uint8_t *buf;
    int64_t sbase;
    uint32_t span;
    uint32_t inside;
    const uint8_t *tail;  // a long pattern's bytes past its first 32 (global), else null
    uint32_t mtail;
};

// The bytes of a long pattern past its first 32 (tail[0..len)) against the
// text at internal position P (inside the text: P + len <= lim), from global
// memory.
__device__ __noinline__ bool verify_tail(const SearchJob &J, int64_t P, const uint8_t *tail,
                                         uint32_t len) {
    for (uint32_t i = 0; i < len; ++i)
        if (ldg_u8(J.base + P + i) != ldg_u8(tail + i)) return false;
    return true;
}

// t[P..P+m) == p, read from the staged bytes when they cover it (shared
// memory word loads), else from global memory.
__device__ __forceinline__ bool verify_staged(const SearchJob &J, int64_t P, const StagedText &T) {
    const int64_t o = P - T.sbase;
    const uint32_t m = J.pat.m;
    if (T.inside && o >= 0 && o + (int64_t)m <= (int64_t)T.span) {
        const uint32_t *W = reinterpret_cast<const uint32_t *>(T.buf);
        const uint32_t a = (uint32_t)o >> 2, sh = ((uint32_t)o & 3u) * 8u;
        const uint32_t nw = (m + 3u) >> 2;
        uint32_t cur = W[a];
        for (uint32_t i = 0; i < nw; ++i) {
            const uint32_t nxt = W[a + i + 1u];
            if ((__funnelshift_r(cur, nxt, sh) ^ J.pat.w[i]) & word_mask(m, i)) return false;
            cur = nxt;
        }
        return true;
    }
    return verify_global(J, P);
}

// The text's bytes [P+m-8, P+m) against p's last 8 bytes (m >= 8), read from
// the staged bytes when they cover them, else from global memory.  With P-q
// an occurrence and q <= 8 a period of p, this decides whether P is one.
__device__ __forceinline__ bool tail8_ok(const SearchJob &J, int64_t P, const StagedText &T) {
    const int64_t a = P + (int64_t)J.pat.m - 8;
    const int64_t o = a - T.sbase;
    uint32_t x0, x1, x2;
    const uint32_t sh = ((uint32_t)a & 3u) * 8u;
    if (T.inside && o >= 0 && o + 8 <= (int64_t)T.span) {
        const uint32_t *W = reinterpret_cast<const uint32_t *>(T.buf);
        const uint32_t wa = (uint32_t)o >> 2;  // (sbase is 16-byte aligned)
        x0 = W[wa];
        x1 = W[wa + 1];
        x2 = sh ? W[wa + 2] : 0u;
    } else {
        const uint64_t wa = (uint64_t)a >> 2;
        x0 = load_word(J, wa);
        x1 = load_word(J, wa + 1);
        x2 = sh ? load_word(J, wa + 2) : 0u;
    }
    return __funnelshift_r(x0, x1, sh) == J.pat.tl && __funnelshift_r(x1, x2, sh) == J.pat.th;
}

// ---------------------------------------------------------------------------
// warp scans
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t t = __shfl_up_sync(kFull, v, d);
        if (lane >= d) v += t;
    }
    return v;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}

__device__ __forceinline__ uint64_t warp_sum64(uint64_t v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}

}  // namespace epsm
